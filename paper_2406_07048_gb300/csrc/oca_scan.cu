// The step-2 LQ problem of the ADMM (Sec. IV-B, one SQP QP per iteration)
// solved for a batch of independent problems, in two forms:
//
//   OCA_LQ_SCAN        parallel in time.  The optimality conditions link each
//                      stage's state and costate lam_t = dV_t/ds_t linearly,
//                        s_{t+1} = A_t s_t + b_t - C_t lam_{t+1},
//                        lam_t   = J_t s_t - eta_t + A_t^T lam_{t+1},
//                      with b_t = c_t - B_t R_t^-1 r_t, C_t = B_t R_t^-1 B_t^T,
//                      J_t = Q_t, eta_t = -q_t, and lam_N = Q_N s_N + q_N as the
//                      element (0, 0, 0, Q_N, -q_N).  Two consecutive relations
//                      compose into one of the same form (eliminating the shared
//                      state and costate, M = (I + C1 J2)^-1):
//                        A = A2 M A1,  b = A2 M (b1 + C1 eta2) + b2,
//                        C = A2 M C1 A2^T + C2,  J = J1 + A1^T M^T J2 A1,
//                        eta = eta1 + A1^T M^T (eta2 - J2 b1),
//                      an associative operation, so every suffix e_t o ... o e_N
//                      (whose A is 0: lam_t = J s_t - eta, the value function
//                      P_t = J, p_t = -eta) is formed in ceil(log2(N + 1)) rounds
//                      in which element t takes element t + 2^r, one CTA per
//                      composition.  The gains K_t, k_t follow per stage in
//                      parallel, and the rollout s_{t+1} = (A + B K) s + B k + c
//                      is a dependent chain of matrix-vector products (one warp).
//   OCA_LQ_SEQUENTIAL  the backward Riccati recursion over t (one CTA per
//                      problem), then the same gains and rollout.
//
// FP64 throughout.  One CTA per composition: its two elements, the augmented
// systems [I + C1 J2 | A1, b1 + C1 eta2, C1 A2^T] and [I + J2 C1 | J2 A1,
// eta2 - J2 b1] (the second matrix is the transpose of the first: C1, J2 are
// symmetric) live in shared memory and are reduced by Gauss-Jordan elimination
// with partial pivoting.
#include <cfloat>

#include "oca_common.cuh"
#include "oca_kernels.h"

namespace oca {

constexpr int kLqMaxS = 12;  // state dimension
constexpr int kLqMaxU = 4;   // input dimension

struct LqArgs {
    int n, m, N, S;              // state, input, horizon, problems
    const double *A, *B, *c;     // [S][N][n][n], [S][N][n][m], [S][N][n]
    const double *Q, *q;         // [S][N+1][n][n], [S][N+1][n]
    const double *R, *r;         // [S][N][m][m], [S][N][m]
    const double *s0;            // [S][n]
    double *s, *u;               // [S][N+1][n], [S][N][m]
    double *P, *p;               // [S][N+1][n][n], [S][N+1][n] or null
    int *status;                 // [S]: 0 solved, 1 singular or non-finite
    double *buf0, *buf1;         // element buffers [S][N+1][es]
    double *F, *f, *K, *k;       // closed-loop maps and gains [S][N][..]
};

__host__ __device__ inline int lq_es(int n) { return 3 * n * n + 2 * n; }

// small dense inverse by Gauss-Jordan with partial pivoting (every caller
// thread computes it in registers); false if a pivot is not above `tiny`
__device__ inline bool small_inverse(double (&M)[kLqMaxU][kLqMaxU], double (&X)[kLqMaxU][kLqMaxU], int m) {
    double W[kLqMaxU][2 * kLqMaxU];
#pragma unroll
    for (int i = 0; i < kLqMaxU; ++i)
#pragma unroll
        for (int j = 0; j < 2 * kLqMaxU; ++j)
            W[i][j] = j < kLqMaxU ? (i < m && j < m ? M[i][j] : (i == j ? 1.0 : 0.0)) : (i == j - kLqMaxU ? 1.0 : 0.0);
    double amax = 0.0;
#pragma unroll
    for (int i = 0; i < kLqMaxU; ++i)
#pragma unroll
        for (int j = 0; j < kLqMaxU; ++j) amax = fmax(amax, fabs(W[i][j]));
    bool ok = isfinite(amax);
#pragma unroll
    for (int c = 0; c < kLqMaxU; ++c) {
        int pr = c;
        double best = fabs(W[c][c]);
#pragma unroll
        for (int i = c + 1; i < kLqMaxU; ++i)
            if (fabs(W[i][c]) > best) {
                best = fabs(W[i][c]);
                pr = i;
            }
        if (!(best > 1e-300 + 1e-14 * amax)) {
            ok = false;
            best = 1.0;
        }
#pragma unroll
        for (int i = 0; i < kLqMaxU; ++i)
            if (i == pr && pr != c)
#pragma unroll
                for (int j = 0; j < 2 * kLqMaxU; ++j) {
                    const double tmp = W[c][j];
                    W[c][j] = W[i][j];
                    W[i][j] = tmp;
                }
        const double ip = 1.0 / (W[c][c] != 0.0 ? W[c][c] : 1.0);
#pragma unroll
        for (int j = 0; j < 2 * kLqMaxU; ++j) W[c][j] *= ip;
#pragma unroll
        for (int i = 0; i < kLqMaxU; ++i)
            if (i != c) {
                const double fct = W[i][c];
#pragma unroll
                for (int j = 0; j < 2 * kLqMaxU; ++j) W[i][j] -= fct * W[c][j];
            }
    }
#pragma unroll
    for (int i = 0; i < kLqMaxU; ++i)
#pragma unroll
        for (int j = 0; j < kLqMaxU; ++j) X[i][j] = W[i][kLqMaxU + j];
    return ok;
}

// ---- stage elements (one warp per stage and problem)
__global__ void __launch_bounds__(32) k_lq_elem(LqArgs a) {
    const int t = blockIdx.x, s = blockIdx.y, lane = threadIdx.x;
    const int n = a.n, m = a.m, N = a.N, nn = n * n, E = N + 1;
    double *e = a.buf0 + ((size_t)s * E + t) * lq_es(n);
    double *Ae = e, *be = e + nn, *Ce = be + n, *Je = Ce + nn, *he = Je + nn;
    const double *Qt = a.Q + ((size_t)s * E + t) * nn, *qt = a.q + ((size_t)s * E + t) * n;
    for (int k2 = lane; k2 < nn; k2 += 32) Je[k2] = Qt[k2];
    for (int i = lane; i < n; i += 32) he[i] = -qt[i];
    if (t == N) {
        for (int k2 = lane; k2 < nn; k2 += 32) {
            Ae[k2] = 0.0;
            Ce[k2] = 0.0;
        }
        for (int i = lane; i < n; i += 32) be[i] = 0.0;
        return;
    }
    const size_t st = (size_t)s * N + t;
    const double *At = a.A + st * nn, *Bt = a.B + st * n * m, *ct = a.c + st * n;
    const double *Rt = a.R + st * m * m, *rt = a.r + st * m;
    double Rm[kLqMaxU][kLqMaxU], Ri[kLqMaxU][kLqMaxU], z[kLqMaxU];
#pragma unroll
    for (int i = 0; i < kLqMaxU; ++i)
#pragma unroll
        for (int j = 0; j < kLqMaxU; ++j) Rm[i][j] = (i < m && j < m) ? Rt[i * m + j] : 0.0;
    const bool ok = small_inverse(Rm, Ri, m);
    if (!ok && lane == 0) a.status[s] = 1;
#pragma unroll
    for (int i = 0; i < kLqMaxU; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < kLqMaxU; ++j)
            if (i < m && j < m) acc += Ri[i][j] * rt[j];
        z[i] = acc;
    }
    for (int k2 = lane; k2 < nn; k2 += 32) Ae[k2] = At[k2];
    for (int i = lane; i < n; i += 32) {
        double acc = ct[i];
        for (int x = 0; x < m; ++x) acc -= Bt[i * m + x] * z[x];
        be[i] = acc;
    }
    // C = B R^-1 B^T
    for (int k2 = lane; k2 < nn; k2 += 32) {
        const int i = k2 / n, j = k2 % n;
        double acc = 0.0;
        for (int x = 0; x < m; ++x) {
            double w = 0.0;
            for (int y = 0; y < m; ++y) w += Ri[x][y] * Bt[j * m + y];
            acc += Bt[i * m + x] * w;
        }
        Ce[k2] = acc;
    }
}

// ---- one round of compositions: nxt[t] = cur[t] o cur[t + d] (or cur[t])
constexpr int kLqThreads = 128;

__global__ void __launch_bounds__(kLqThreads) k_lq_compose(LqArgs a, const double *cur, double *nxt, int d) {
    const int t = blockIdx.x, s = blockIdx.y, tid = threadIdx.x;
    const int n = a.n, nn = n * n, E = a.N + 1, es = lq_es(n);
    const double *e1g = cur + ((size_t)s * E + t) * es;
    double *eo = nxt + ((size_t)s * E + t) * es;
    if (t + d >= E) {
        for (int k2 = tid; k2 < es; k2 += kLqThreads) eo[k2] = e1g[k2];
        return;
    }
    const double *e2g = cur + ((size_t)s * E + t + d) * es;
    constexpr int MES = 3 * kLqMaxS * kLqMaxS + 2 * kLqMaxS;
    constexpr int WXM = 3 * kLqMaxS + 1, WYM = 2 * kLqMaxS + 1;
    __shared__ double e1[MES], e2[MES], GX[kLqMaxS * WXM], GY[kLqMaxS * WYM], rowx[WXM], rowy[WYM];
    __shared__ int piv[2];
    __shared__ int bad;
    for (int k2 = tid; k2 < es; k2 += kLqThreads) {
        e1[k2] = e1g[k2];
        e2[k2] = e2g[k2];
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    const double *A1 = e1, *b1 = e1 + nn, *C1 = b1 + n, *J1 = C1 + nn, *h1 = J1 + nn;
    const double *A2 = e2, *b2 = e2 + nn, *C2 = b2 + n, *J2 = C2 + nn, *h2 = J2 + nn;
    const int WX = 3 * n + 1, WY = 2 * n + 1;
    // [I + C1 J2 | A1 | b1 + C1 eta2 | C1 A2^T] and [I + J2 C1 | J2 A1 | eta2 - J2 b1]
    for (int k2 = tid; k2 < n * WX; k2 += kLqThreads) {
        const int i = k2 / WX, j = k2 % WX;
        double v;
        if (j < n) {
            v = i == j ? 1.0 : 0.0;
            for (int x = 0; x < n; ++x) v += C1[i * n + x] * J2[x * n + j];
        } else if (j < 2 * n) {
            v = A1[i * n + j - n];
        } else if (j == 2 * n) {
            v = b1[i];
            for (int x = 0; x < n; ++x) v += C1[i * n + x] * h2[x];
        } else {
            const int jj = j - 2 * n - 1;
            v = 0.0;
            for (int x = 0; x < n; ++x) v += C1[i * n + x] * A2[jj * n + x];
        }
        GX[i * WX + j] = v;
    }
    for (int k2 = tid; k2 < n * WY; k2 += kLqThreads) {
        const int i = k2 / WY, j = k2 % WY;
        double v;
        if (j < n) {
            v = i == j ? 1.0 : 0.0;
            for (int x = 0; x < n; ++x) v += J2[i * n + x] * C1[x * n + j];
        } else if (j < 2 * n) {
            v = 0.0;
            for (int x = 0; x < n; ++x) v += J2[i * n + x] * A1[x * n + j - n];
        } else {
            v = h2[i];
            for (int x = 0; x < n; ++x) v -= J2[i * n + x] * b1[x];
        }
        GY[i * WY + j] = v;
    }
    __syncthreads();
    // Gauss-Jordan with partial pivoting on both systems: warp 0 picks GX's
    // pivot, warp 1 GY's (ties to the lower row)
    const int warp = tid >> 5, lane = tid & 31;
    for (int col = 0; col < n; ++col) {
        if (warp < 2) {
            const double *G = warp == 0 ? GX : GY;
            const int W = warp == 0 ? WX : WY;
            double v = -1.0;
            int idx = n;
            if (lane >= col && lane < n) {
                v = fabs(G[lane * W + col]);
                idx = lane;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_down_sync(0xffffffffu, v, o);
                const int i2 = __shfl_down_sync(0xffffffffu, idx, o);
                if (v2 > v || (v2 == v && i2 < idx)) {
                    v = v2;
                    idx = i2;
                }
            }
            if (lane == 0) {
                if (!(v > 1e-300) || idx >= n) {
                    bad = 1;
                    idx = col;
                }
                piv[warp] = idx;
            }
        }
        __syncthreads();
        // swap the pivot row into place and scale it (into the row buffers)
        const int px = piv[0], py = piv[1];
        for (int j = tid; j < WX + WY; j += kLqThreads) {
            if (j < WX) {
                const double a0 = GX[col * WX + j], a1 = GX[px * WX + j];
                GX[px * WX + j] = a0;
                rowx[j] = a1;
            } else {
                const int jj = j - WX;
                const double a0 = GY[col * WY + jj], a1 = GY[py * WY + jj];
                GY[py * WY + jj] = a0;
                rowy[jj] = a1;
            }
        }
        __syncthreads();
        const double ipx = 1.0 / (rowx[col] != 0.0 ? rowx[col] : 1.0);
        const double ipy = 1.0 / (rowy[col] != 0.0 ? rowy[col] : 1.0);
        // eliminate column col from every other row; the pivot row becomes the scaled row
        for (int k2 = tid; k2 < n * (WX + WY); k2 += kLqThreads) {
            const bool isx = k2 < n * WX;
            const int W = isx ? WX : WY;
            const int kk = isx ? k2 : k2 - n * WX;
            const int i = kk / W, j = kk % W;
            if (j <= col) continue;
            double *G = isx ? GX : GY;
            const double rj = (isx ? rowx[j] * ipx : rowy[j] * ipy);
            if (i == col) G[i * W + j] = rj;
            else G[i * W + j] -= G[i * W + col] * rj;
        }
        __syncthreads();
    }
    if (tid == 0 && bad) a.status[s] = 1;
    // X = M [A1 | b1 + C1 eta2 | C1 A2^T] in GX[:, n:], Y = M^T [J2 A1 | eta2 - J2 b1] in GY[:, n:]
    double *Ao = eo, *bo = eo + nn, *Co = bo + n, *Jo = Co + nn, *ho = Jo + nn;
    for (int k2 = tid; k2 < es; k2 += kLqThreads) {
        double v;
        if (k2 < nn) {                       // A = A2 XA
            const int i = k2 / n, j = k2 % n;
            v = 0.0;
            for (int x = 0; x < n; ++x) v += A2[i * n + x] * GX[x * WX + n + j];
            Ao[k2] = v;
        } else if (k2 < nn + n) {            // b = A2 Xb + b2
            const int i = k2 - nn;
            v = b2[i];
            for (int x = 0; x < n; ++x) v += A2[i * n + x] * GX[x * WX + 2 * n];
            bo[i] = v;
        } else if (k2 < 2 * nn + n) {        // C = A2 XC + C2
            const int kk = k2 - nn - n, i = kk / n, j = kk % n;
            v = C2[kk];
            for (int x = 0; x < n; ++x) v += A2[i * n + x] * GX[x * WX + 2 * n + 1 + j];
            Co[kk] = v;
        } else if (k2 < 3 * nn + n) {        // J = J1 + A1^T YJ
            const int kk = k2 - 2 * nn - n, i = kk / n, j = kk % n;
            v = J1[kk];
            for (int x = 0; x < n; ++x) v += A1[x * n + i] * GY[x * WY + n + j];
            Jo[kk] = v;
        } else {                             // eta = eta1 + A1^T Ye
            const int i = k2 - 3 * nn - n;
            v = h1[i];
            for (int x = 0; x < n; ++x) v += A1[x * n + i] * GY[x * WY + 2 * n];
            ho[i] = v;
        }
    }
}

// ---- gains of stage t from the value function of stage t + 1:
//   K = -(R + B^T P B)^-1 B^T P A,  k = -(R + B^T P B)^-1 (B^T (P c + p) + r),
// and the closed-loop map s_{t+1} = F s_t + f, F = A + B K, f = c + B k.
// Block t = N (and every t) also writes the value functions when requested.
// vf: the elements whose J, -eta are P_t, p_t (sequential form: null, P/p given)
__global__ void __launch_bounds__(64) k_lq_gains(LqArgs a, const double *vf, const double *Pv, const double *pv) {
    const int t = blockIdx.x, s = blockIdx.y, tid = threadIdx.x;
    const int n = a.n, m = a.m, N = a.N, nn = n * n, E = N + 1, es = lq_es(n);
    auto Pat = [&](int tt, int k2) -> double {
        return vf ? vf[((size_t)s * E + tt) * es + 2 * nn + n + k2] : Pv[((size_t)s * E + tt) * nn + k2];
    };
    auto pat = [&](int tt, int i) -> double {
        return vf ? -vf[((size_t)s * E + tt) * es + 3 * nn + n + i] : pv[((size_t)s * E + tt) * n + i];
    };
    if (vf && a.P)
        for (int k2 = tid; k2 < nn; k2 += 64) a.P[((size_t)s * E + t) * nn + k2] = Pat(t, k2);
    if (vf && a.p)
        for (int i = tid; i < n; i += 64) a.p[((size_t)s * E + t) * n + i] = pat(t, i);
    if (t == N) return;
    __shared__ double P[kLqMaxS * kLqMaxS], pp[kLqMaxS], PB[kLqMaxS * kLqMaxU], w[kLqMaxS], H[kLqMaxU * kLqMaxS],
        g[kLqMaxU], Kt[kLqMaxU * kLqMaxS], kt[kLqMaxU];
    const size_t st = (size_t)s * N + t;
    const double *At = a.A + st * nn, *Bt = a.B + st * n * m, *ct = a.c + st * n;
    const double *Rt = a.R + st * m * m, *rt = a.r + st * m;
    for (int k2 = tid; k2 < nn; k2 += 64) P[k2] = Pat(t + 1, k2);
    for (int i = tid; i < n; i += 64) pp[i] = pat(t + 1, i);
    __syncthreads();
    for (int k2 = tid; k2 < n * m + n; k2 += 64) {
        if (k2 < n * m) {
            const int i = k2 / m, x = k2 % m;
            double v = 0.0;
            for (int y = 0; y < n; ++y) v += P[i * n + y] * Bt[y * m + x];
            PB[k2] = v;
        } else {
            const int i = k2 - n * m;
            double v = pp[i];
            for (int y = 0; y < n; ++y) v += P[i * n + y] * ct[y];
            w[i] = v;                                  // P c + p
        }
    }
    __syncthreads();
    for (int k2 = tid; k2 < m * n + m; k2 += 64) {
        if (k2 < m * n) {
            const int x = k2 / n, j = k2 % n;
            double v = 0.0;
            for (int y = 0; y < n; ++y) v += PB[y * m + x] * At[y * n + j];
            H[k2] = v;                                 // B^T P A
        } else {
            const int x = k2 - m * n;
            double v = rt[x];
            for (int y = 0; y < n; ++y) v += Bt[y * m + x] * w[y];
            g[x] = v;                                  // B^T (P c + p) + r
        }
    }
    __syncthreads();
    double Sm[kLqMaxU][kLqMaxU], Si[kLqMaxU][kLqMaxU];
#pragma unroll
    for (int x = 0; x < kLqMaxU; ++x)
#pragma unroll
        for (int y = 0; y < kLqMaxU; ++y) {
            double v = 0.0;
            if (x < m && y < m) {
                v = Rt[x * m + y];
                for (int l = 0; l < n; ++l) v += Bt[l * m + x] * PB[l * m + y];
            }
            Sm[x][y] = v;
        }
    const bool ok = small_inverse(Sm, Si, m);
    if (!ok && tid == 0) a.status[s] = 1;
    for (int k2 = tid; k2 < m * n + m; k2 += 64) {
        const int x = k2 < m * n ? k2 / n : k2 - m * n;
        double v = 0.0;
        for (int y = 0; y < m; ++y) v -= Si[x][y] * (k2 < m * n ? H[y * n + k2 % n] : g[y]);
        if (k2 < m * n) Kt[k2] = v;
        else kt[x] = v;
    }
    __syncthreads();
    double *Ko = a.K + st * m * n, *ko = a.k + st * m, *Fo = a.F + st * nn, *fo = a.f + st * n;
    for (int k2 = tid; k2 < m * n + m; k2 += 64) {
        if (k2 < m * n) Ko[k2] = Kt[k2];
        else ko[k2 - m * n] = kt[k2 - m * n];
    }
    for (int k2 = tid; k2 < nn + n; k2 += 64) {
        if (k2 < nn) {
            const int i = k2 / n, j = k2 % n;
            double v = At[k2];
            for (int x = 0; x < m; ++x) v += Bt[i * m + x] * Kt[x * n + j];
            Fo[k2] = v;
        } else {
            const int i = k2 - nn;
            double v = ct[i];
            for (int x = 0; x < m; ++x) v += Bt[i * m + x] * kt[x];
            fo[i] = v;
        }
    }
}

// ---- rollout s_{t+1} = F_t s_t + f_t (one warp per problem: lane i owns s_i;
// the next stage's row of F is loaded while the current one is applied),
// then u_t = K_t s_t + k_t
__global__ void __launch_bounds__(32) k_lq_rollout(LqArgs a) {
    const int s = blockIdx.x, lane = threadIdx.x;
    const int n = a.n, N = a.N, nn = n * n;
    const bool own = lane < n;
    double x = own ? a.s0[(size_t)s * n + lane] : 0.0;
    if (own) a.s[(size_t)s * (N + 1) * n + lane] = x;
    double row[kLqMaxS], nrow[kLqMaxS], fv = 0.0, nf = 0.0;
    const double *F0 = a.F + (size_t)s * N * nn, *f0 = a.f + (size_t)s * N * n;
#pragma unroll
    for (int k2 = 0; k2 < kLqMaxS; ++k2) row[k2] = (N > 0 && own && k2 < n) ? F0[lane * n + k2] : 0.0;
    if (N > 0 && own) fv = f0[lane];
    for (int t = 0; t < N; ++t) {
        const bool more = t + 1 < N;
#pragma unroll
        for (int k2 = 0; k2 < kLqMaxS; ++k2)
            nrow[k2] = (more && own && k2 < n) ? F0[(size_t)(t + 1) * nn + lane * n + k2] : 0.0;
        if (more && own) nf = f0[(size_t)(t + 1) * n + lane];
        double v = fv;
#pragma unroll
        for (int k2 = 0; k2 < kLqMaxS; ++k2) v += row[k2] * __shfl_sync(0xffffffffu, x, k2);
        x = v;
        if (own) a.s[((size_t)s * (N + 1) + t + 1) * n + lane] = x;
#pragma unroll
        for (int k2 = 0; k2 < kLqMaxS; ++k2) row[k2] = nrow[k2];
        fv = nf;
    }
}

__global__ void __launch_bounds__(32) k_lq_controls(LqArgs a) {
    const int t = blockIdx.x, s = blockIdx.y, lane = threadIdx.x;
    const int n = a.n, m = a.m, N = a.N;
    if (lane >= m) return;
    const size_t st = (size_t)s * N + t;
    const double *Kt = a.K + st * m * n, *xt = a.s + ((size_t)s * (N + 1) + t) * n;
    double v = a.k[st * m + lane];
    for (int j = 0; j < n; ++j) v += Kt[lane * n + j] * xt[j];
    a.u[st * m + lane] = v;
}

// ---- sequential backward Riccati recursion (one CTA per problem):
//   Quu = R + B^T P B, Qus = B^T P A, qu = B^T (P c + p) + r,
//   Qss = Q + A^T P A, qs = q + A^T (P c + p), K = -Quu^-1 Qus, k = -Quu^-1 qu,
//   P_t = Qss + Qus^T K, p_t = qs + Qus^T k;  P_N = Q_N, p_N = q_N.
// The value functions go to Pv, pv; the gains kernel then forms K, k, F, f.
__global__ void __launch_bounds__(kLqThreads) k_lq_seq(LqArgs a, double *Pv, double *pv) {
    const int s = blockIdx.x, tid = threadIdx.x;
    const int n = a.n, m = a.m, N = a.N, nn = n * n, E = N + 1;
    __shared__ double P[kLqMaxS * kLqMaxS], pp[kLqMaxS], PA[kLqMaxS * kLqMaxS], PB[kLqMaxS * kLqMaxU],
        w[kLqMaxS], H[kLqMaxU * kLqMaxS], g[kLqMaxU], Kt[kLqMaxU * kLqMaxS], kt[kLqMaxU];
    __shared__ int bad;
    if (tid == 0) bad = 0;
    const double *QN = a.Q + ((size_t)s * E + N) * nn, *qN = a.q + ((size_t)s * E + N) * n;
    for (int k2 = tid; k2 < nn; k2 += kLqThreads) {
        P[k2] = QN[k2];
        Pv[((size_t)s * E + N) * nn + k2] = QN[k2];
    }
    for (int i = tid; i < n; i += kLqThreads) {
        pp[i] = qN[i];
        pv[((size_t)s * E + N) * n + i] = qN[i];
    }
    __syncthreads();
    for (int t = N - 1; t >= 0; --t) {
        const size_t st = (size_t)s * N + t;
        const double *At = a.A + st * nn, *Bt = a.B + st * n * m, *ct = a.c + st * n;
        const double *Rt = a.R + st * m * m, *rt = a.r + st * m;
        const double *Qt = a.Q + ((size_t)s * E + t) * nn, *qt = a.q + ((size_t)s * E + t) * n;
        // PA, PB, w = P c + p
        for (int k2 = tid; k2 < nn + n * m + n; k2 += kLqThreads) {
            if (k2 < nn) {
                const int i = k2 / n, j = k2 % n;
                double v = 0.0;
                for (int y = 0; y < n; ++y) v += P[i * n + y] * At[y * n + j];
                PA[k2] = v;
            } else if (k2 < nn + n * m) {
                const int kk = k2 - nn, i = kk / m, x = kk % m;
                double v = 0.0;
                for (int y = 0; y < n; ++y) v += P[i * n + y] * Bt[y * m + x];
                PB[kk] = v;
            } else {
                const int i = k2 - nn - n * m;
                double v = pp[i];
                for (int y = 0; y < n; ++y) v += P[i * n + y] * ct[y];
                w[i] = v;
            }
        }
        __syncthreads();
        // Qus = B^T P A, qu = B^T w + r
        for (int k2 = tid; k2 < m * n + m; k2 += kLqThreads) {
            if (k2 < m * n) {
                const int x = k2 / n, j = k2 % n;
                double v = 0.0;
                for (int y = 0; y < n; ++y) v += Bt[y * m + x] * PA[y * n + j];
                H[k2] = v;
            } else {
                const int x = k2 - m * n;
                double v = rt[x];
                for (int y = 0; y < n; ++y) v += Bt[y * m + x] * w[y];
                g[x] = v;
            }
        }
        __syncthreads();
        double Sm[kLqMaxU][kLqMaxU], Si[kLqMaxU][kLqMaxU];
#pragma unroll
        for (int x = 0; x < kLqMaxU; ++x)
#pragma unroll
            for (int y = 0; y < kLqMaxU; ++y) {
                double v = 0.0;
                if (x < m && y < m) {
                    v = Rt[x * m + y];
                    for (int l = 0; l < n; ++l) v += Bt[l * m + x] * PB[l * m + y];
                }
                Sm[x][y] = v;
            }
        if (!small_inverse(Sm, Si, m) && tid == 0) bad = 1;
        for (int k2 = tid; k2 < m * n + m; k2 += kLqThreads) {
            const int x = k2 < m * n ? k2 / n : k2 - m * n;
            double v = 0.0;
            for (int y = 0; y < m; ++y) v -= Si[x][y] * (k2 < m * n ? H[y * n + k2 % n] : g[y]);
            if (k2 < m * n) Kt[k2] = v;
            else kt[x] = v;
        }
        __syncthreads();
        // P_t = Q + A^T P A + Qus^T K, p_t = q + A^T w + Qus^T k (upper triangle, mirrored)
        for (int k2 = tid; k2 < nn + n; k2 += kLqThreads) {
            if (k2 < nn) {
                const int i = k2 / n, j = k2 % n;
                if (j < i) continue;
                double v = Qt[k2];
                for (int y = 0; y < n; ++y) v += At[y * n + i] * PA[y * n + j];
                for (int x = 0; x < m; ++x) v += H[x * n + i] * Kt[x * n + j];
                P[i * n + j] = v;
                P[j * n + i] = v;
            } else {
                const int i = k2 - nn;
                double v = qt[i];
                for (int y = 0; y < n; ++y) v += At[y * n + i] * w[y];
                for (int x = 0; x < m; ++x) v += H[x * n + i] * kt[x];
                pp[i] = v;
            }
        }
        __syncthreads();
        for (int k2 = tid; k2 < nn; k2 += kLqThreads) Pv[((size_t)s * E + t) * nn + k2] = P[k2];
        for (int i = tid; i < n; i += kLqThreads) pv[((size_t)s * E + t) * n + i] = pp[i];
        __syncthreads();
    }
    if (tid == 0 && bad) a.status[s] = 1;
}

__global__ void k_lq_reset(int *status, int S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S) status[i] = 0;
}

// workspace: two element buffers (scan) or the value functions (sequential),
// then K, k, F, f; every region 256-byte aligned
struct LqWork {
    size_t buf0, buf1, K, k, F, f, bytes;
};

static LqWork lq_work(int n, int m, int N, int S) {
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    LqWork w;
    const size_t E = (size_t)N + 1;
    size_t o = 0;
    w.buf0 = o;
    o += al(sizeof(double) * (size_t)S * E * lq_es(n));
    w.buf1 = o;
    o += al(sizeof(double) * (size_t)S * E * lq_es(n));
    w.K = o;
    o += al(sizeof(double) * (size_t)S * N * m * n);
    w.k = o;
    o += al(sizeof(double) * (size_t)S * N * m);
    w.F = o;
    o += al(sizeof(double) * (size_t)S * N * n * n);
    w.f = o;
    o += al(sizeof(double) * (size_t)S * N * n);
    w.bytes = o;
    return w;
}

size_t lq_workspace_bytes(int n, int m, int N, int S) { return lq_work(n, m, N, S).bytes; }

cudaError_t launch_lq(int method, int n, int m, int N, int S, const double *A, const double *B, const double *c,
                      const double *Q, const double *q, const double *R, const double *r, const double *s0, double *s,
                      double *u, double *P, double *p, int *status, void *work, cudaStream_t st) {
    const LqWork w = lq_work(n, m, N, S);
    unsigned char *wb = static_cast<unsigned char *>(work);
    LqArgs a;
    a.n = n;
    a.m = m;
    a.N = N;
    a.S = S;
    a.A = A;
    a.B = B;
    a.c = c;
    a.Q = Q;
    a.q = q;
    a.R = R;
    a.r = r;
    a.s0 = s0;
    a.s = s;
    a.u = u;
    a.P = P;
    a.p = p;
    a.status = status;
    a.buf0 = reinterpret_cast<double *>(wb + w.buf0);
    a.buf1 = reinterpret_cast<double *>(wb + w.buf1);
    a.K = reinterpret_cast<double *>(wb + w.K);
    a.k = reinterpret_cast<double *>(wb + w.k);
    a.F = reinterpret_cast<double *>(wb + w.F);
    a.f = reinterpret_cast<double *>(wb + w.f);
    const int E = N + 1;
    k_lq_reset<<<(S + 255) / 256, 256, 0, st>>>(status, S);
    if (method == 0) {
        k_lq_elem<<<dim3(E, S), 32, 0, st>>>(a);
        double *cur = a.buf0, *nxt = a.buf1;
        for (int d = 1; d < E; d *= 2) {
            k_lq_compose<<<dim3(E, S), kLqThreads, 0, st>>>(a, cur, nxt, d);
            double *sw = cur;
            cur = nxt;
            nxt = sw;
        }
        k_lq_gains<<<dim3(E, S), 64, 0, st>>>(a, cur, nullptr, nullptr);
    } else {
        // value functions into the first buffer region (S * E * (n^2 + n) doubles fit in it)
        double *Pv = a.buf0, *pv = a.buf0 + (size_t)S * E * n * n;
        k_lq_seq<<<S, kLqThreads, 0, st>>>(a, Pv, pv);
        k_lq_gains<<<dim3(E, S), 64, 0, st>>>(a, nullptr, Pv, pv);
        if (P) {
            cudaError_t e = cudaMemcpyAsync(P, Pv, sizeof(double) * (size_t)S * E * n * n, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        }
        if (p) {
            cudaError_t e = cudaMemcpyAsync(p, pv, sizeof(double) * (size_t)S * E * n, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        }
    }
    k_lq_rollout<<<S, 32, 0, st>>>(a);
    if (N > 0) k_lq_controls<<<dim3(N, S), 32, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace oca

using namespace oca;

extern "C" oca_status oca_lq_workspace_bytes(int32_t ns, int32_t nu, int32_t N, int32_t n_problems, int64_t *bytes) {
    if (!bytes || ns < 1 || nu < 1 || N < 0 || n_problems < 1) return OCA_ERR_INVALID_ARGUMENT;
    if (ns > kLqMaxS || nu > kLqMaxU || N > OCA_MAX_LQ_HORIZON || n_problems > 65535) return OCA_ERR_CAPACITY;
    *bytes = (int64_t)lq_workspace_bytes(ns, nu, N, n_problems);
    return OCA_OK;
}

extern "C" oca_status oca_lq_solve(oca_ctx *ctx, int32_t method, int32_t ns, int32_t nu, int32_t N, int32_t n_problems,
                                   const double *A, const double *B, const double *c, const double *Q, const double *q,
                                   const double *R, const double *r, const double *s0, double *s, double *u, double *P,
                                   double *p, int32_t *status, void *work, int64_t work_bytes, void *stream) {
    if (!ctx || (method != OCA_LQ_SCAN && method != OCA_LQ_SEQUENTIAL)) return OCA_ERR_INVALID_ARGUMENT;
    if (ns < 1 || nu < 1 || N < 0 || n_problems < 1) return OCA_ERR_INVALID_ARGUMENT;
    if (ns > kLqMaxS || nu > kLqMaxU || N > OCA_MAX_LQ_HORIZON || n_problems > 65535) return OCA_ERR_CAPACITY;
    if (!Q || !q || !s0 || !s || !status || !work) return OCA_ERR_INVALID_ARGUMENT;
    if (N > 0 && (!A || !B || !c || !R || !r || !u)) return OCA_ERR_INVALID_ARGUMENT;
    if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return OCA_ERR_INVALID_ARGUMENT;
    if (work_bytes < (int64_t)lq_workspace_bytes(ns, nu, N, n_problems)) return OCA_ERR_CAPACITY;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaError_t e = launch_lq(method == OCA_LQ_SCAN ? 0 : 1, ns, nu, N, n_problems, A, B, c, Q, q, R, r, s0, s,
                                    u, P, p, status, work, st);
    return e == cudaSuccess ? OCA_OK : OCA_ERR_CUDA;
}
