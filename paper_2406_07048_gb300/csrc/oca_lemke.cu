// The paper's own pair-QP solver on the GPU (Sec. IV-C), as a comparison
// kernel for the semismooth Newton solver of the hot path: the pair QP
// eqn:const_least_square with y_e eliminated through its equality
// (eqn:const_least_square_ineq), the KKT conditions (eqn:kkt_conditions)
// written as the LCP w = M z + q, w, z >= 0, w^T z = 0
// (eqn:linear_complementarity_problem), solved by Lemke's complementary
// pivoting with one thread per LCP row, as the paper parallelises it.
//
// One warp per pair, lane i owning LCP row i (L <= 32 rows).  Revised form:
// each lane keeps its row of B^-1 (the tableau's w columns) in shared memory;
// the entering column is B^-1 times the original column, the ratio test a
// warp reduction with the lexicographic rule (columns of B^-1) on ties.
#include <cfloat>

#include "oca_common.cuh"
#include "oca_kernels.h"

namespace oca {


__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <typename T>
__device__ __forceinline__ T big_value() { return sizeof(T) == sizeof(float) ? T(FLT_MAX) : T(DBL_MAX); }

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// scenario of pair p (binary search over the scenarios' first pairs)
__device__ __forceinline__ int pair_scenario(const ScenMeta *meta, int S, long long p) {
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (meta[mid].pair0 <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T, int D>
__global__ void __launch_bounds__(128) k_lemke(LemkeArgs<T> a) {
    constexpr int V = D + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wid = threadIdx.x >> 5, lane = lane_id();
    const long long p = (long long)blockIdx.x * (blockDim.x >> 5) + wid;
    if (p >= a.P) return;
    T *Msh = reinterpret_cast<T *>(smem_raw) + (size_t)wid * 32 * 65;  // M [32][32], Binv [32][33]
    T *Bi = Msh + 32 * 32;
    __shared__ T Krow[4][32][4];  // generators of the warp's pair (rows <= 32, V <= 4), per warp
    __shared__ T rowr[4][33];     // the pivot row of B^-1 and its rhs, per warp

    // ---- the pair: scenario, (j, part, t), pose, geometry
    const int s = pair_scenario(a.meta, a.n_scen, p);
    const ScenMeta sm = a.meta[s];
    const long long r = p - sm.pair0;
    const int N = sm.N, NP = sm.NP;
    const int t = (int)(r % N) + 1, part = (int)((r / N) % NP), j = (int)(r / ((long long)N * NP));
    const int gp = sm.part0 + part, gm = sm.obs0 + j;
    const int col = sm.qbeg + part * N + (t - 1);
    const int nr = a.g.part_nf[gp], no = a.g.obs_nf[gm], ny = nr + no + 1;
    const int FR = a.g.FR, FO = a.g.FO;
    const long long P = a.P;
    T rho[D], R[D * D];
#pragma unroll
    for (int i = 0; i < D; ++i) rho[i] = a.pose[(long long)i * a.Qtot + col];
#pragma unroll
    for (int i = 0; i < D * D; ++i) R[i] = a.pose[(long long)(D + i) * a.Qtot + col];
    // generator rows K_g (body frame) and kappa_g, lane g
    T Kg[V], kap = T(0), ybar = T(0);
#pragma unroll
    for (int c = 0; c < V; ++c) Kg[c] = T(0);
    if (lane < nr) {
#pragma unroll
        for (int i = 0; i < D; ++i) Kg[1 + i] = a.g.part_A[((long long)gp * FR + lane) * D + i];
        kap = a.g.part_b[(long long)gp * FR + lane];
        ybar = a.y_in[(long long)lane * P + p];
    } else if (lane < nr + no) {
        const int m = lane - nr;
        T c[D], cr = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            c[i] = a.g.obs_C[((long long)gm * FO + m) * D + i];
            cr += c[i] * rho[i];
        }
        Kg[0] = a.g.obs_d[(long long)gm * FO + m] - cr;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            T acc = T(0);
#pragma unroll
            for (int l = 0; l < D; ++l) acc += R[l * D + i] * c[l];
            Kg[1 + i] = acc;
        }
        ybar = a.y_in[(long long)(FR + m) * P + p];
    } else if (lane == nr + no) {
        Kg[0] = T(1);
        ybar = a.y_in[(long long)(FR + FO) * P + p];
    }
    T Dg = T(0);
#pragma unroll
    for (int c = 0; c < V; ++c) Dg += Kg[c] * Kg[c];
    // eliminated component: the robot face with the largest b (lowest index on ties)
    int e = 0;
    {
        T bb = __shfl_sync(0xffffffffu, kap, 0);
        for (int k = 1; k < nr; ++k) {
            const T bk = __shfl_sync(0xffffffffu, kap, k);
            if (bk > bb) {
                bb = bk;
                e = k;
            }
        }
    }
    const T ke = __shfl_sync(0xffffffffu, kap, e), De = __shfl_sync(0xffffffffu, Dg, e);
    const T ybe = __shfl_sync(0xffffffffu, ybar, e);
    T Ke[V];
#pragma unroll
    for (int c = 0; c < V; ++c) Ke[c] = __shfl_sync(0xffffffffu, Kg[c], e);
    // remaining components u: lane a of the LCP owns component (a < e ? a : a + 1)
    const int n = ny - 1, L = n + 1;
    const int src = lane < e ? lane : lane + 1;
    T Ku[V];
#pragma unroll
    for (int c = 0; c < V; ++c) Ku[c] = __shfl_sync(0xffffffffu, Kg[c], src & 31);
    const T ku = __shfl_sync(0xffffffffu, kap, src & 31), Du = __shfl_sync(0xffffffffu, Dg, src & 31);
    const T ybu = __shfl_sync(0xffffffffu, ybar, src & 31);
    const T eta_t = T(1) / ke;
    const T kt = ku / ke;                               // kappa~ = kappa_u / kappa_e
    T Kt[V], bt[V];
#pragma unroll
    for (int c = 0; c < V; ++c) {
        Kt[c] = Ku[c] - kt * Ke[c];                     // K~ = K_u - kappa~ K_e
        const T bqc = c == 0 ? T(1) + a.zeta[p] : a.xi[(long long)(c - 1) * P + p];
        bt[c] = bqc + Ke[c] * eta_t;                    // b~ = bq + K_e eta / kappa_e
    }
    if (lane < n) {
#pragma unroll
        for (int c = 0; c < V; ++c) Krow[wid][lane][c] = Kt[c];
    }
    __syncwarp();
    // LCP: M = [[H, kt], [-kt^T, 0]], q = [f; eta~]; H = K~ K~^T + prox (diag D_u + D_e kt kt^T)
    const T kt_all = kt;
    T q = T(0);
    if (lane < n) {
        for (int c2 = 0; c2 < n; ++c2) {
            T h = T(0);
#pragma unroll
            for (int c = 0; c < V; ++c) h += Kt[c] * Krow[wid][c2][c];
            const T kt2 = __shfl_sync(__activemask(), kt_all, c2);
            if (a.prox > T(0)) h += a.prox * ((c2 == lane ? Du : T(0)) + De * kt * kt2);
            Msh[lane * 32 + c2] = h;
        }
        Msh[lane * 32 + n] = kt;
        T f = T(0);
#pragma unroll
        for (int c = 0; c < V; ++c) f += Kt[c] * bt[c];
        if (a.prox > T(0)) f += a.prox * (-De * kt * (eta_t - ybe) - Du * ybu);
        q = f;
    }
    __syncwarp();
    if (lane < n) Msh[n * 32 + lane] = -Msh[lane * 32 + n];
    if (lane == n) {
        Msh[n * 32 + n] = T(0);
        q = eta_t;
    }
    // ---- Lemke: variables w_i (id i), z_i (id L + i), z0 (id 2L)
    for (int k = 0; k < 33; ++k) Bi[lane * 33 + k] = T(0);
    if (lane < L) Bi[lane * 33 + lane] = T(1);
    __syncwarp();
    // Pivots are chosen on q + delta, delta a small generic perturbation (a
    // numerical stand-in for the symbolic one of the lexicographic rule,
    // which floating-point ties defeat on degenerate LCPs); the basic
    // variables are recomputed from the final B^-1 with the original q.
    T qabs = lane < L ? m_abs(q) : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qabs = fmax(qabs, __shfl_xor_sync(0xffffffffu, qabs, o));
    const T frac = T(0.7548776662466927) * T(lane + 1) - floor(T(0.7548776662466927) * T(lane + 1));
    const T qp = lane < L ? q + (sizeof(T) == sizeof(float) ? T(1e-5) : T(1e-9)) * (T(1) + qabs) * (T(0.5) + frac) : T(0);
    T rhs = qp;
    int basis = lane;
    int status = OCA_PAIR_OK;
    const T qmin = warp_min(lane < L ? q : big_value<T>());
    if (qmin < T(0)) {
        // first pivot: z0 enters, the row of the most negative q leaves (largest index on ties)
        const T qpmin = warp_min(lane < L ? qp : big_value<T>());
        unsigned ties = __ballot_sync(0xffffffffu, lane < L && qp <= qpmin);
        int rr = 31 - __clz(ties);
        int enter = 2 * L;
        int leaving = -1;
        for (int piv = 0; piv < 50 * L + 50; ++piv) {
            // entering column c = B^-1 x (original column of `enter`)
            T cval = T(0);
            if (lane < L) {
                if (enter < L) {
                    cval = Bi[lane * 33 + enter];
                } else if (enter < 2 * L) {
                    const int jz = enter - L;
                    for (int k = 0; k < L; ++k) cval -= Bi[lane * 33 + k] * Msh[k * 32 + jz];
                } else {
                    for (int k = 0; k < L; ++k) cval -= Bi[lane * 33 + k];
                }
            }
            if (piv > 0) {
                // minimum ratio over rows with a positive entry; ties by the
                // lexicographic rule on the rows of B^-1 / c, z0 preferred
                T cmax = lane < L ? m_abs(cval) : T(0);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
                const T ctol = T(64) * m_eps<T>() * (T(1) + cmax);
                const bool elig = lane < L && cval > ctol;
                const T ratio = elig ? rhs / cval : big_value<T>();
                const T th = warp_min(ratio);
                if (!(th < big_value<T>())) {
                    status = OCA_PAIR_DEGENERATE;  // ray termination
                    break;
                }
                unsigned cand = __ballot_sync(0xffffffffu, elig && ratio <= th + T(64) * m_eps<T>() * (T(1) + m_abs(th)));
                const unsigned z0c = __ballot_sync(0xffffffffu, elig && basis == 2 * L) & cand;
                if (z0c) {
                    cand = z0c;
                } else {
                    for (int k = 0; k < L && __popc(cand) > 1; ++k) {
                        const bool in = (cand >> lane) & 1u;
                        const T v = in ? Bi[lane * 33 + k] / cval : big_value<T>();
                        const T mn = warp_min(v);
                        cand &= __ballot_sync(0xffffffffu, in && v <= mn + T(64) * m_eps<T>() * (T(1) + m_abs(mn)));
                    }
                }
                rr = __ffs(cand) - 1;
            }
            // pivot on (rr, enter)
            const T cr = __shfl_sync(0xffffffffu, cval, rr);
            leaving = __shfl_sync(0xffffffffu, basis, rr);
            if (lane == rr) {
                const T ic = T(1) / cr;
                for (int k = 0; k < L; ++k) {
                    const T v = Bi[lane * 33 + k] * ic;
                    Bi[lane * 33 + k] = v;
                    rowr[wid][k] = v;
                }
                rhs *= ic;
                rowr[wid][32] = rhs;
                basis = enter;
            }
            __syncwarp();
            if (lane != rr && lane < L) {
                for (int k = 0; k < L; ++k) Bi[lane * 33 + k] -= cval * rowr[wid][k];
                rhs -= cval * rowr[wid][32];
            }
            __syncwarp();
            if (leaving == 2 * L) break;  // z0 left the basis: complementary solution
            enter = leaving < L ? leaving + L : leaving - L;
            if (piv == 50 * L + 49) status = OCA_PAIR_ITER_CAP;
        }
        if (status == OCA_PAIR_OK && leaving != 2 * L) status = OCA_PAIR_ITER_CAP;
        if (status == OCA_PAIR_OK) {
            // exact basic values on the final basis: x_B = B^-1 q
            T xb = T(0);
            for (int k = 0; k < L; ++k) xb += Bi[lane * 33 + k] * __shfl_sync(0xffffffffu, q, k);
            const bool neg = lane < L && xb < -T(64) * m_eps<T>() * (T(1) + qabs) * T(L);
            if (!__any_sync(0xffffffffu, neg)) rhs = xb;
        }
    }
    // z of the basic z columns; y_u = z[0..n), y_e = eta~ - kt . y_u
    T zl = (basis >= L && basis < 2 * L) ? fmax(T(0), rhs) : T(0);
    // scatter z to lanes by index: lane a needs z_a
    T za = T(0);
    for (int i = 0; i < L; ++i) {
        const int bi = __shfl_sync(0xffffffffu, basis, i);
        const T zi = __shfl_sync(0xffffffffu, zl, i);
        if (bi == L + lane) za = zi;
    }
    T kz = lane < n ? kt * za : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kz += __shfl_xor_sync(0xffffffffu, kz, o);
    const T ye = eta_t - kz;
    // y of generator g (lane g): g == e -> ye, else z of LCP index (g < e ? g : g - 1)
    const int ai = lane < e ? lane : lane - 1;
    const T zg = __shfl_sync(0xffffffffu, za, ai & 31);
    const T yg = lane == e ? ye : zg;
    if (lane < ny) {
        const int comp = lane < nr ? lane : (lane < nr + no ? FR + lane - nr : FR + FO);
        a.y_out[(long long)comp * P + p] = yg;
    }
    // v = K^T y + bq, objective
    T vv[V];
#pragma unroll
    for (int c = 0; c < V; ++c) {
        T acc = lane < ny ? Kg[c] * yg : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        vv[c] = acc + (c == 0 ? T(1) + a.zeta[p] : a.xi[(long long)(c - 1) * P + p]);
    }
    if (lane == 0) {
        T o = T(0);
#pragma unroll
        for (int c = 0; c < V; ++c) {
            if (a.v_out) a.v_out[(long long)c * P + p] = vv[c];
            o += T(0.5) * vv[c] * vv[c];
        }
        if (a.obj_out) a.obj_out[p] = o;
        if (a.status_out) a.status_out[p] = status;
    }
}

template <typename T>
cudaError_t launch_lemke(const LemkeArgs<T> &a, int dim, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    const int warps = 4;
    const size_t sm = (size_t)warps * 32 * 65 * sizeof(T);
    const unsigned blocks = (unsigned)((a.P + warps - 1) / warps);
    cudaError_t e;
    if (dim == 2) {
        if (sm > 48 * 1024 && (e = cudaFuncSetAttribute(k_lemke<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
            return e;
        k_lemke<T, 2><<<blocks, 32 * warps, sm, st>>>(a);
    } else {
        if (sm > 48 * 1024 && (e = cudaFuncSetAttribute(k_lemke<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
            return e;
        k_lemke<T, 3><<<blocks, 32 * warps, sm, st>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t launch_lemke<float>(const LemkeArgs<float> &, int, cudaStream_t);
template cudaError_t launch_lemke<double>(const LemkeArgs<double> &, int, cudaStream_t);

}  // namespace oca
