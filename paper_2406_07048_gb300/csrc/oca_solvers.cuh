// Per-pair solvers, callable from device and host code:
//   - the pair QP of Sec. IV-C (eqn:const_least_square) by a primal
//     active-set / minimum-norm-point method (prox = 0) or by semismooth
//     Newton on its (D+1)-dimensional dual (prox > 0);
//   - the scale LP of Sec. III-A (eqn:scale_opt) through its dual
//     (eqn:scale_opt_dual) by a revised two-phase simplex.
// Host compilation exists so that the same code can be exercised off-GPU.
#pragma once

#include <cfloat>
#include <cmath>

#include "oca_common.cuh"

namespace oca {

// ============================================================================
// per-lane problem data
// ============================================================================
template <typename T, int D>
struct Lane {
    T rho[D], R[D * D];  // pose of the part
    const T *A, *b;      // part halfspaces (body frame), stride D
    int nr;
    const T *C, *d;      // obstacle halfspaces (world frame)
    int no;
};

// Generator g of the pair QP (rows of K, Sec. IV-C), with lambda rescaled to
// lambda_hat = b * lambda so that the equality becomes sum(lambda_hat) = 1:
//   g < nr       : [0; a_g / b_g]
//   g < nr + no  : [d'_m; c'_m] = [d_m - c_m.rho; R^T c_m]
//   g = nr + no  : [1; 0]  (slack gamma)
template <typename T, int D>
OCA_HD inline void gen_vec(const Lane<T, D> &L, int g, T out[D + 1]) {
    if (g < L.nr) {
        const T ib = T(1) / ldg(L.b + g);
        out[0] = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) out[1 + i] = ldg(L.A + g * D + i) * ib;
    } else if (g < L.nr + L.no) {
        const int m = g - L.nr;
        T c[D];
#pragma unroll
        for (int i = 0; i < D; ++i) c[i] = ldg(L.C + m * D + i);
        T cr = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) cr += c[i] * L.rho[i];
        out[0] = ldg(L.d + m) - cr;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) acc += L.R[k * D + i] * c[k];
            out[1 + i] = acc;
        }
    } else {
        out[0] = T(1);
#pragma unroll
        for (int i = 0; i < D; ++i) out[1 + i] = T(0);
    }
}

template <typename T, int V>
OCA_HD inline T dotv(const T *a, const T *b) {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < V; ++i) s += a[i] * b[i];
    return s;
}

// world-frame vector u = R v1 - v0 rho: <v, [d'_m; c'_m]> = v0 d_m + c_m . u
template <typename T, int D>
OCA_HD inline void world_dir(const Lane<T, D> &L, const T v[D + 1], T u[D]) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T acc = -v[0] * L.rho[i];
#pragma unroll
        for (int k = 0; k < D; ++k) acc += L.R[i * D + k] * v[1 + k];
        u[i] = acc;
    }
}

// Small symmetric positive-definite solve (n <= NMAX) by Cholesky; G is
// lower-triangular-used, overwritten.  Returns false if not positive definite.
template <typename T, int NMAX>
OCA_HD inline bool chol_solve(T G[NMAX][NMAX], T r[NMAX], int n, T tiny) {
    // G = L L^T with the reciprocal of each diagonal entry kept (one
    // reciprocal square root per column instead of a square root and a
    // division per use)
    T il[NMAX];
#pragma unroll
    for (int a = 0; a < NMAX; ++a) {
        il[a] = T(0);
        if (a < n) {
            T dgn = G[a][a];
#pragma unroll
            for (int k = 0; k < NMAX; ++k)
                if (k < a) dgn -= G[a][k] * G[a][k];
            if (!(dgn > tiny)) return false;
            const T ia = m_rsqrt(dgn);
            il[a] = ia;
            G[a][a] = dgn * ia;
#pragma unroll
            for (int b2 = 0; b2 < NMAX; ++b2) {
                if (b2 > a && b2 < n) {
                    T acc = G[b2][a];
#pragma unroll
                    for (int k = 0; k < NMAX; ++k)
                        if (k < a) acc -= G[b2][k] * G[a][k];
                    G[b2][a] = acc * ia;
                }
            }
        }
    }
#pragma unroll
    for (int a = 0; a < NMAX; ++a) {
        if (a < n) {
            T acc = r[a];
#pragma unroll
            for (int k = 0; k < NMAX; ++k)
                if (k < a) acc -= G[a][k] * r[k];
            r[a] = acc * il[a];
        }
    }
#pragma unroll
    for (int a = NMAX - 1; a >= 0; --a) {
        if (a < n) {
            T acc = r[a];
#pragma unroll
            for (int k = 0; k < NMAX; ++k)
                if (k > a && k < n) acc -= G[k][a] * r[k];
            r[a] = acc * il[a];
        }
    }
    return true;
}

// ============================================================================
// Pair QP, prox = 0: primal active-set / minimum-norm-point method.
//   min |v|^2,  v = bq + sum lambda_hat_k p_k + sum mu_m q_m + gamma e0,
//   sum lambda_hat = 1, all weights >= 0.
// The support S (at most D+2 generators, affinely independent) carries the
// weights; a major cycle adds the generator most violating the optimality
// conditions (<v, p_k> = min over the lambda hull, <v, q_m> >= 0), minor
// cycles restore positivity by a line search towards the affine minimiser.
// ============================================================================
template <typename T, int D>
struct Support {
    int n;
    int id[D + 2];
    T w[D + 2];
};

template <typename T, int D>
OCA_HD inline void sup_point(const Lane<T, D> &L, const Support<T, D> &S, const T bq[D + 1], T v[D + 1],
                             T *vscale = nullptr) {
    T sc = T(0);
#pragma unroll
    for (int i = 0; i <= D; ++i) {
        v[i] = bq[i];
        sc += m_abs(bq[i]);
    }
#pragma unroll
    for (int k = 0; k < D + 2; ++k) {
        if (k < S.n) {
            T g[D + 1];
            gen_vec<T, D>(L, S.id[k], g);
#pragma unroll
            for (int i = 0; i <= D; ++i) {
                v[i] += S.w[k] * g[i];
                sc += m_abs(S.w[k] * g[i]);
            }
        }
    }
    if (vscale) *vscale = sc;
}

// Affine minimiser of |v|^2 over the affine hull of S (lambda weights sum to 1).
template <typename T, int D>
OCA_HD bool sup_affine(const Lane<T, D> &L, const Support<T, D> &S, const T bq[D + 1], T wn[D + 2]) {
    constexpr int V = D + 1, SM = D + 2;
    int ib = -1;
#pragma unroll
    for (int k = SM - 1; k >= 0; --k)
        if (k < S.n && S.id[k] < L.nr) ib = k;
    if (ib < 0) return false;
    T gb[V];
    int idb = 0;
#pragma unroll
    for (int k = 0; k < SM; ++k)
        if (k == ib) idb = S.id[k];
    gen_vec<T, D>(L, idb, gb);
    T x0[V];
#pragma unroll
    for (int i = 0; i < V; ++i) x0[i] = bq[i] + gb[i];
    T dir[V][V];
    int slot[V];
    bool isl[V];
    int m = 0;
#pragma unroll
    for (int k = 0; k < SM; ++k) {
        if (k < S.n && k != ib) {
            T g[V];
            gen_vec<T, D>(L, S.id[k], g);
            const bool lam = S.id[k] < L.nr;
#pragma unroll
            for (int a = 0; a < V; ++a) {
                if (a == m) {
#pragma unroll
                    for (int i = 0; i < V; ++i) dir[a][i] = lam ? g[i] - gb[i] : g[i];
                    slot[a] = k;
                    isl[a] = lam;
                }
            }
            ++m;
        }
    }
    if (m > V) return false;
    // least squares min |x0 + Dir t| by modified Gram-Schmidt QR of the
    // directions (twice-orthogonalised), which keeps the conditioning of
    // nearly parallel generators (distant obstacles) instead of squaring it
    T Qm[V][V], Rm[V][V], r[V];
#pragma unroll
    for (int a = 0; a < V; ++a) {
        if (a < m) {
            T nrm0 = T(0);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                Qm[a][i] = dir[a][i];
                nrm0 += dir[a][i] * dir[a][i];
            }
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
                for (int b2 = 0; b2 < V; ++b2) {
                    if (b2 < a) {
                        const T c = dotv<T, V>(Qm[b2], Qm[a]);
                        if (pass == 0) Rm[b2][a] = c; else Rm[b2][a] += c;
#pragma unroll
                        for (int i = 0; i < V; ++i) Qm[a][i] -= c * Qm[b2][i];
                    }
                }
            }
            const T nrm = m_sqrt(dotv<T, V>(Qm[a], Qm[a]));
            if (!(nrm > T(32) * m_eps<T>() * m_sqrt(nrm0))) return false;
            Rm[a][a] = nrm;
#pragma unroll
            for (int i = 0; i < V; ++i) Qm[a][i] /= nrm;
            r[a] = -dotv<T, V>(Qm[a], x0);
        }
    }
#pragma unroll
    for (int a = V - 1; a >= 0; --a) {
        if (a < m) {
            T acc = r[a];
#pragma unroll
            for (int b2 = 0; b2 < V; ++b2)
                if (b2 > a && b2 < m) acc -= Rm[a][b2] * r[b2];
            r[a] = acc / Rm[a][a];
        }
    }
    T sl = T(0);
#pragma unroll
    for (int k = 0; k < SM; ++k) wn[k] = T(0);
#pragma unroll
    for (int a = 0; a < V; ++a) {
        if (a < m) {
#pragma unroll
            for (int k = 0; k < SM; ++k)
                if (k == slot[a]) wn[k] = r[a];
            if (isl[a]) sl += r[a];
        }
    }
#pragma unroll
    for (int k = 0; k < SM; ++k)
        if (k == ib) wn[k] = T(1) - sl;
    return true;
}

// remove entries with weight <= wtol (stable compaction, static indexing)
template <typename T, int D>
OCA_HD inline void sup_compact(Support<T, D> &S, T wtol) {
    constexpr int SM = D + 2;
    int n = 0;
    int id2[SM];
    T w2[SM];
#pragma unroll
    for (int k = 0; k < SM; ++k) {
        id2[k] = 0;
        w2[k] = T(0);
    }
#pragma unroll
    for (int k = 0; k < SM; ++k) {
        if (k < S.n && S.w[k] > wtol) {
#pragma unroll
            for (int j = 0; j < SM; ++j)
                if (j == n) {
                    id2[j] = S.id[k];
                    w2[j] = S.w[k];
                }
            ++n;
        }
    }
    S.n = n;
#pragma unroll
    for (int k = 0; k < SM; ++k) {
        S.id[k] = id2[k];
        S.w[k] = w2[k];
    }
}

template <typename T, int D>
OCA_HD inline bool sup_has(const Support<T, D> &S, int g) {
    bool h = false;
#pragma unroll
    for (int k = 0; k < D + 2; ++k) h |= (k < S.n && S.id[k] == g);
    return h;
}

template <typename T, int D>
OCA_HD void sup_cold(const Lane<T, D> &L, const T bq[D + 1], Support<T, D> &S) {
    // best single vertex of the lambda hull
    int best = 0;
    T bv = T(0);
    for (int k = 0; k < L.nr; ++k) {
        T g[D + 1];
        gen_vec<T, D>(L, k, g);
        T v2 = T(0);
#pragma unroll
        for (int i = 0; i <= D; ++i) v2 += (bq[i] + g[i]) * (bq[i] + g[i]);
        if (k == 0 || v2 < bv) {
            bv = v2;
            best = k;
        }
    }
    S.n = 1;
    S.id[0] = best;
    S.w[0] = T(1);
#pragma unroll
    for (int k = 1; k < D + 2; ++k) {
        S.id[k] = 0;
        S.w[k] = T(0);
    }
}

// Minor cycles: move S to a positive affine minimiser.  Returns false on a
// singular working set.
template <typename T, int D>
OCA_HD bool mnp_minor(const Lane<T, D> &L, Support<T, D> &S, const T bq[D + 1], int newest, bool &dropped_newest_at_zero) {
    constexpr int SM = D + 2;
    dropped_newest_at_zero = false;
    for (int mc = 0; mc < SM + 1; ++mc) {
        T wn[SM];
        if (!sup_affine<T, D>(L, S, bq, wn)) return false;
        T wmax = T(1);
#pragma unroll
        for (int k = 0; k < SM; ++k)
            if (k < S.n) wmax = fmax(wmax, m_abs(wn[k]));
        const T wtol = T(8) * m_eps<T>() * wmax;
        bool allpos = true;
#pragma unroll
        for (int k = 0; k < SM; ++k)
            if (k < S.n && !(wn[k] > wtol)) allpos = false;
        if (allpos) {
#pragma unroll
            for (int k = 0; k < SM; ++k)
                if (k < S.n) S.w[k] = wn[k];
            return true;
        }
        T theta = T(1);
        int drop = -1;
#pragma unroll
        for (int k = 0; k < SM; ++k) {
            if (k < S.n && !(wn[k] > wtol)) {
                const T den = S.w[k] - wn[k];
                const T th = den > T(0) ? S.w[k] / den : T(0);
                if (th < theta || drop < 0) {
                    theta = th;
                    drop = k;
                }
            }
        }
        theta = fmax(T(0), fmin(theta, T(1)));
        int dropid = -1;
#pragma unroll
        for (int k = 0; k < SM; ++k) {
            if (k < S.n) {
                S.w[k] += theta * (wn[k] - S.w[k]);
                if (k == drop) {
                    dropid = S.id[k];
                    S.w[k] = T(0);
                }
            }
        }
        if (dropid == newest && theta <= T(0)) dropped_newest_at_zero = true;
        sup_compact<T, D>(S, wtol);
        if (dropped_newest_at_zero) return true;
    }
    return true;
}

template <typename T, int D>
OCA_HD int mnp_solve(const Lane<T, D> &L, Support<T, D> &S, const T bq[D + 1], T v[D + 1]) {
    constexpr int V = D + 1, SM = D + 2;
    const int ng = L.nr + L.no + 1;
    const T tol = T(32) * m_eps<T>();
    int status = OCA_PAIR_OK;
    bool dz;
    if (!mnp_minor<T, D>(L, S, bq, -1, dz)) {
        sup_cold<T, D>(L, bq, S);  // warm start was singular
    }
    const int cap = 4 * ng + 8;
    int it = 0;
    for (; it < cap; ++it) {
        T vscale;
        sup_point<T, D>(L, S, bq, v, &vscale);
        // v at rounding level of its own terms: the global minimum 0 is reached
        T vn = T(0);
#pragma unroll
        for (int i = 0; i <= D; ++i) vn += v[i] * v[i];
        if (m_sqrt(vn) <= T(64) * m_eps<T>() * vscale) break;
        // nu = <v, x_lambda>, the common value on the lambda support
        T nu = T(0);
#pragma unroll
        for (int k = 0; k < SM; ++k) {
            if (k < S.n && S.id[k] < L.nr) {
                T g[V];
                gen_vec<T, D>(L, S.id[k], g);
                nu += S.w[k] * dotv<T, V>(v, g);
            }
        }
        T vn1 = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) vn1 += v[1 + i] * v[1 + i];
        vn1 = m_sqrt(vn1);
        T u[D];
        world_dir<T, D>(L, v, u);
        T best = T(0);
        int bi = -1;
        for (int k = 0; k < L.nr; ++k) {
            const T ib = T(1) / ldg(L.b + k);
            T h = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) h += ldg(L.A + k * D + i) * v[1 + i];
            h = h * ib - nu;
            const T scale = vn1 * ib + m_abs(nu) + T(1e-30);
            if (h < -tol * scale && h < best && !sup_has<T, D>(S, k)) {
                best = h;
                bi = k;
            }
        }
        for (int m = 0; m < L.no; ++m) {
            const T dm = ldg(L.d + m);
            T h = v[0] * dm, cr = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const T c = ldg(L.C + m * D + i);
                h += c * u[i];
                cr += c * L.rho[i];
            }
            const T scale = m_abs(v[0]) * (m_abs(dm) + m_abs(cr)) + vn1 + T(1e-30);
            if (h < -tol * scale && h < best && !sup_has<T, D>(S, L.nr + m)) {
                best = h;
                bi = L.nr + m;
            }
        }
        {
            const T h = v[0];
            if (h < -tol * (m_abs(v[0]) + vn1 + T(1e-30)) && h < best && !sup_has<T, D>(S, L.nr + L.no)) {
                best = h;
                bi = L.nr + L.no;
            }
        }
        if (bi < 0) break;  // optimal
        // A full support spans the whole space, so its affine minimiser is
        // v = 0: a remaining violation is rounding noise (optimal).
        if (S.n >= SM) break;
        Support<T, D> keep = S;
#pragma unroll
        for (int k = 0; k < SM; ++k)
            if (k == S.n) {
                S.id[k] = bi;
                S.w[k] = T(0);
            }
        S.n += 1;
        if (!mnp_minor<T, D>(L, S, bq, bi, dz)) {
            // the entering generator lies in the affine hull of S to rounding:
            // its violation was rounding noise, S is optimal
            S = keep;
            break;
        }
        if (dz) break;  // the new generator could not enter: converged to rounding
    }
    if (it >= cap) status = OCA_PAIR_ITER_CAP;
    sup_point<T, D>(L, S, bq, v);
    return status;
}

// ============================================================================
// Pair QP, prox > 0: semismooth Newton on the (D+1)-dimensional dual.
//   min 0.5|K^T y + bq|^2 + 0.5 rho sum_g |K_g|^2 (y_g - ybar_g)^2,
//   y in Y = {y >= 0, b^T lambda = 1}  (y unscaled: generators [0; a_k], kappa = b)
// The proximal metric Dg = |K_g|^2 measures each generator's step in
// residual space.  The minimiser is y(w) = P_Y^D(ybar - Dg^-1 K w / rho)
// (projection in the Dg metric) at the unique root w of
//   F(w) = w - bq - K^T y(w)   (w = v* = K^T y* + bq).
// F is the gradient of the strongly convex
//   psi(w) = 0.5|w|^2 - bq.w - [0.5 rho |y(w) - ybar|_D^2 + (K w).y(w)]
// and piecewise affine, with generalised Jacobian
//   I + sum_active K_g K_g^T / (rho |K_g|^2)  (minus the simplex correction),
// whose conditioning is bounded by 1 + n/rho whatever the obstacle offsets;
// Newton steps with an Armijo search on psi terminate finitely.
// ============================================================================
template <typename T, int D>
struct SsnState {
    T tau;       // simplex threshold of the lambda projection
    T Kty[D + 1];
    T psi;
    T H[D + 1][D + 1];  // rho I + K^T P D^-1 K  (full)
    T mag;       // sum |K_g| y_g: rounding scale of K^T y
    T pmag;      // sum of the magnitudes of psi's terms: rounding scale of psi
};

// lambda_k = max(0, z_k - tau b_k / D_k) with sum_k b_k lambda_k = 1:
// breakpoints t_k = z_k D_k / b_k, on the active set tau = (sum b z - 1) / sum b^2/D.
template <typename T>
OCA_HD inline T simplex_tau(const T *z, const T *b, const T *Dk, int nr) {
    T tau = T(0);
    int best_n = -1;
#pragma unroll
    for (int k = 0; k < kMaxFR; ++k) {
        if (k < nr) {
            const T tk = z[k] * Dk[k] / b[k];
            T s1 = T(0), s2 = T(0);
            int n = 0;
#pragma unroll
            for (int j = 0; j < kMaxFR; ++j) {
                if (j < nr && z[j] * Dk[j] / b[j] >= tk) {
                    s1 += b[j] * z[j];
                    s2 += b[j] * b[j] / Dk[j];
                    ++n;
                }
            }
            const T tc = (s1 - T(1)) / s2;
            if (tc < tk && n > best_n) {
                best_n = n;
                tau = tc;
            }
        }
    }
    return tau;
}

template <typename T, int D>
OCA_HD inline void ssn_eval(const Lane<T, D> &L, const T *ybar, long long P, int FR, int FO, T rho_p,
                           const T bq[D + 1], const T w[D + 1], bool want_H, SsnState<T, D> &st) {
    constexpr int V = D + 1;
    T zl[kMaxFR], bl[kMaxFR], dl[kMaxFR];
#pragma unroll
    for (int k = 0; k < kMaxFR; ++k) {
        if (k < L.nr) {
            T h = T(0), a2 = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const T ai = ldg(L.A + k * D + i);
                h += ai * w[1 + i];
                a2 += ai * ai;
            }
            bl[k] = ldg(L.b + k);
            dl[k] = a2;
            zl[k] = ybar[(long long)k * P] - h / (rho_p * a2);
        } else {
            zl[k] = T(0);
            bl[k] = T(1);
            dl[k] = T(1);
        }
    }
    const T tau = simplex_tau<T>(zl, bl, dl, L.nr);
    st.tau = tau;
    T pen = T(0), lin = T(0), mag = T(0);
    T a1[D], sc[D], sd = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        a1[i] = T(0);
        sc[i] = T(0);
    }
    // lambda part of K^T P D^-1 K: sum_A p p^T / D - (sum_A b p / D)(...)^T / sum_A b^2 / D
    T Ha[D][D], ba[D], bb = T(0);
    if (want_H) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            ba[i] = T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) Ha[i][k] = T(0);
        }
    }
#pragma unroll
    for (int k = 0; k < kMaxFR; ++k) {
        if (k < L.nr) {
            const T lk = fmax(T(0), zl[k] - tau * bl[k] / dl[k]);
            const T yb = ybar[(long long)k * P];
            T ak[D];
#pragma unroll
            for (int i = 0; i < D; ++i) ak[i] = ldg(L.A + k * D + i);
            T h = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) h += ak[i] * w[1 + i];
            pen += dl[k] * (lk - yb) * (lk - yb);
            lin += h * lk;
#pragma unroll
            for (int i = 0; i < D; ++i) a1[i] += lk * ak[i];
            mag += lk;
            if (want_H && lk > T(0)) {
                const T id = T(1) / dl[k];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    ba[i] += bl[k] * ak[i] * id;
#pragma unroll
                    for (int j = 0; j < D; ++j) Ha[i][j] += ak[i] * ak[j] * id;
                }
                bb += bl[k] * bl[k] * id;
            }
        }
    }
    // R w1: <[d'_m; R^T c_m], w> = w0 d'_m + c_m . (R w1)
    T Rw[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) acc += L.R[i * D + k] * w[1 + k];
        Rw[i] = acc;
    }
    T lmag = m_abs(lin);
    // cone part in world coordinates: Mw = sum_active [d; c][d; c]^T / |K_m|^2
    T Mw[V][V];
    if (want_H) {
#pragma unroll
        for (int i = 0; i < V; ++i)
#pragma unroll
            for (int j = 0; j < V; ++j) Mw[i][j] = T(0);
    }
    for (int m = 0; m < L.no; ++m) {
        T c[D];
        const T dm = ldg(L.d + m);
        T cr = T(0), c2 = T(0), cw = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            c[i] = ldg(L.C + m * D + i);
            cr += c[i] * L.rho[i];
            c2 += c[i] * c[i];
            cw += c[i] * Rw[i];
        }
        const T dp = dm - cr;       // body-frame offset d'_m
        const T h = w[0] * dp + cw;
        const T Dm = dp * dp + c2;  // |[d'_m; R^T c_m]|^2
        const T yb = ybar[(long long)(FR + m) * P];
        const T mu = fmax(T(0), yb - h / (rho_p * Dm));
        pen += Dm * (mu - yb) * (mu - yb);
        lin += h * mu;
        lmag += (m_abs(w[0] * dp) + m_abs(cw)) * mu;
        sd += mu * dp;
#pragma unroll
        for (int i = 0; i < D; ++i) sc[i] += mu * c[i];
        mag += mu * (m_abs(dp) + T(1));
        if (want_H && mu > T(0)) {
            T e[V];
            e[0] = dm;
#pragma unroll
            for (int i = 0; i < D; ++i) e[1 + i] = c[i];
            const T id = T(1) / Dm;
#pragma unroll
            for (int i = 0; i < V; ++i)
#pragma unroll
                for (int j = 0; j < V; ++j) Mw[i][j] += e[i] * e[j] * id;
        }
    }
    const T ybg = ybar[(long long)(FR + FO) * P];
    const T gam = fmax(T(0), ybg - w[0] / rho_p);
    pen += (gam - ybg) * (gam - ybg);
    lin += w[0] * gam;
    mag += gam;
    // K^T y = [sum mu d' + gamma; sum lambda a + R^T sum mu c]
    st.Kty[0] = sd + gam;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T acc = a1[i];
#pragma unroll
        for (int k = 0; k < D; ++k) acc += L.R[k * D + i] * sc[k];
        st.Kty[1 + i] = acc;
    }
    T ww = T(0), bw = T(0);
#pragma unroll
    for (int i = 0; i < V; ++i) {
        ww += w[i] * w[i];
        bw += bq[i] * w[i];
    }
    st.psi = T(0.5) * ww - bw - (T(0.5) * rho_p * pen + lin);
    st.mag = mag;
    st.pmag = T(0.5) * ww + m_abs(bw) + T(0.5) * rho_p * pen + lmag + m_abs(w[0] * gam);
    if (want_H) {
        // H = rho I + Tp Mw Tp^T + e0 e0^T [gamma active] + lambda part,
        // Tp = [[1, -rho^T], [0, R^T]] maps [d_m; c_m] to [d'_m; c'_m].
        T Tp[V][V];
#pragma unroll
        for (int i = 0; i < V; ++i)
#pragma unroll
            for (int j = 0; j < V; ++j) Tp[i][j] = T(0);
        Tp[0][0] = T(1);
#pragma unroll
        for (int j = 0; j < D; ++j) Tp[0][1 + j] = -L.rho[j];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) Tp[1 + i][1 + j] = L.R[j * D + i];
        T TM[V][V];
#pragma unroll
        for (int i = 0; i < V; ++i)
#pragma unroll
            for (int j = 0; j < V; ++j) {
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < V; ++k) acc += Tp[i][k] * Mw[k][j];
                TM[i][j] = acc;
            }
#pragma unroll
        for (int i = 0; i < V; ++i)
#pragma unroll
            for (int j = 0; j < V; ++j) {
                T acc = (i == j) ? rho_p : T(0);
#pragma unroll
                for (int k = 0; k < V; ++k) acc += TM[i][k] * Tp[j][k];
                st.H[i][j] = acc;
            }
        if (gam > T(0)) st.H[0][0] += T(1);
        const T ibb = bb > T(0) ? T(1) / bb : T(0);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) st.H[1 + i][1 + j] += Ha[i][j] - ba[i] * ba[j] * ibb;
    }
}

template <typename T, int D>
OCA_HD inline int ssn_solve(const Lane<T, D> &L, const T *ybar, long long P, int FR, int FO, T rho_p,
                           const T bq[D + 1], T w[D + 1], SsnState<T, D> &st) {
    constexpr int V = D + 1;
    ssn_eval<T, D>(L, ybar, P, FR, FO, rho_p, bq, w, true, st);
    int status = OCA_PAIR_ITER_CAP;
    for (int it = 0; it < 60; ++it) {
        T F[V], fn = T(0), scale = T(1) + st.mag;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            F[i] = w[i] - bq[i] - st.Kty[i];
            fn = fmax(fn, m_abs(F[i]));
            scale = fmax(scale, fmax(m_abs(w[i]), m_abs(bq[i])));
        }
        if (fn <= T(16) * m_eps<T>() * scale) {
            status = OCA_PAIR_OK;
            break;
        }
        if (!(fn == fn)) {
            status = OCA_PAIR_NONFINITE;
            break;
        }
        // Newton direction: (rho I + K^T P D^-1 K) dlt = -rho F
        T G[V][V], dlt[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            dlt[i] = -rho_p * F[i];
#pragma unroll
            for (int j = 0; j < V; ++j) G[i][j] = st.H[i][j];
        }
        if (!chol_solve<T, V>(G, dlt, V, T(0))) {
#pragma unroll
            for (int i = 0; i < V; ++i) dlt[i] = -F[i];
        }
        T gd = T(0);
#pragma unroll
        for (int i = 0; i < V; ++i) gd += F[i] * dlt[i];
        if (!(gd < T(0))) {
#pragma unroll
            for (int i = 0; i < V; ++i) dlt[i] = -F[i];
            gd = T(0);
#pragma unroll
            for (int i = 0; i < V; ++i) gd -= F[i] * F[i];
        }
        T t = T(1);
        SsnState<T, D> trial;
        T wt[V];
        bool ok = false;
        for (int ls = 0; ls < 30; ++ls) {
#pragma unroll
            for (int i = 0; i < V; ++i) wt[i] = w[i] + t * dlt[i];
            ssn_eval<T, D>(L, ybar, P, FR, FO, rho_p, bq, wt, true, trial);
            const T slack = T(8) * m_eps<T>() * (st.pmag + trial.pmag);
            if (trial.psi <= st.psi + T(1e-4) * t * gd + slack && (trial.psi < st.psi || -t * gd <= slack)) {
                ok = true;
                break;
            }
            t *= T(0.5);
        }
#pragma unroll
        for (int i = 0; i < V; ++i) w[i] = wt[i];
        st = trial;
        if (!ok) {
            // no decrease at rounding level: converged as far as the precision allows
            status = OCA_PAIR_OK;
            break;
        }
    }
    return status;
}

// value of generator g's component in the SSN solution; u = R w1
template <typename T, int D>
OCA_HD inline T ssn_value(const Lane<T, D> &L, const T *ybar, long long P, int FR, int FO, T rho_p,
                          const T w[D + 1], const T u[D], T tau, int g) {
    if (g < L.nr) {
        T h = T(0), a2 = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const T ai = ldg(L.A + g * D + i);
            h += ai * w[1 + i];
            a2 += ai * ai;
        }
        return fmax(T(0), ybar[(long long)g * P] - h / (rho_p * a2) - tau * ldg(L.b + g) / a2);
    } else if (g < L.nr + L.no) {
        const int m = g - L.nr;
        // u holds R w1 here: <[d'_m; R^T c_m], w> = w0 d'_m + c_m . (R w1)
        T cr = T(0), c2 = T(0), cw = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const T c = ldg(L.C + m * D + i);
            cr += c * L.rho[i];
            c2 += c * c;
            cw += c * u[i];
        }
        const T dp = ldg(L.d + m) - cr;
        const T h = w[0] * dp + cw;
        return fmax(T(0), ybar[(long long)(FR + m) * P] - h / (rho_p * (dp * dp + c2)));
    }
    return fmax(T(0), ybar[(long long)(FR + FO) * P] - w[0] / rho_p);
}

// ============================================================================
// Semismooth Newton with staged face records (the form the pair kernel runs).
//
// The dual variable is carried in world coordinates, w = [w0; u] with
// u = R w1 (w1 the body-frame part of ssn_solve's variable, R the part's
// rotation).  R is orthogonal, so this is ssn_solve's iteration rotated:
// every generator becomes a world-frame vector -- robot face k: [0; R a_k],
// obstacle face m: [d'_m; c_m] with d'_m = d_m - c_m.rho, slack: [1; 0] --
// and bq = [1 + zeta; R xi].
//
// Per lane (one (part, t) column, fixed over the obstacle sweep) the rotated
// robot normals and the robot constants sit in registers.  Per pair, each
// obstacle face is staged once as the record [d'_m, iD_m, s_m, ybar_m] with
// iD_m = 1 / (prox |K_m|^2) and s_m = ybar_m prox |K_m|^2, and its world
// normal c_m is read from the warp's shared copy of the obstacle's
// halfspaces; an evaluation of y(w) is one pass of multiply-adds over the
// faces: h_m = w0 d'_m + c_m.u, mu_m = max(0, (s_m - h_m) iD_m).
//
// Up to a constant independent of w, the dual function is
//   psi(w) = 0.5 |w|^2 - bq.w + 0.5 sum_m mu_m^2 / iD_m + 0.5 prox gamma^2
//            + 0.5 sum_k prox |a_k|^2 lambda_k^2 + prox tau
// (a face's minimum over y >= 0 of h y + 0.5 prox |K|^2 (y - ybar)^2 is
// 0.5 prox |K|^2 (ybar^2 - mu^2); the robot faces' minimum over
// {lambda >= 0, b.lambda = 1}, with prox tau the multiplier of the equality,
// is sum_k 0.5 prox |a_k|^2 (ybar_k^2 - lambda_k^2) - prox tau), and its
// gradient is F(w) = w - bq - K^T y(w).  psi is convex and piecewise
// quadratic: where the sets of positive lambda, mu and gamma are fixed, F is
// affine with Jacobian H / prox.  A full Newton step from w whose end point
// has the same sets as w therefore lands on the root of F (up to rounding),
// and the solve stops there.
// ============================================================================

// One staged obstacle face of one lane: [d'_m, iD_m, s_m, ybar_m], 16-byte
// aligned (FP32) or 32-byte (FP64).  A lane's records are contiguous; lanes
// are face_lane_stride elements apart, an odd number of 16-byte units, so
// that the eight lanes of each phase of a 16-byte shared load hit distinct
// banks.
template <typename T>
OCA_HD inline int face_lane_stride(int FO) {
    return sizeof(T) == 4 ? 4 * (FO | 1) : 4 * FO + 2;
}
// Normals of an obstacle in the warp's shared buffer: D values per face,
// padded to NrmStride (2 in 2-D, 4 in 3-D) for aligned vector loads; the D
// offsets d_m follow the FO normals.
template <int D>
struct NrmStride {
    static constexpr int N = D == 2 ? 2 : 4;
};
// Elements of one obstacle's buffer, rounded up to 4 (16-byte alignment in
// FP32, 32-byte in FP64).
template <int D>
OCA_HD inline int obs_buf_elems(int FO) {
    return (FO * (NrmStride<D>::N + 1) + 3) & ~3;
}

template <typename T>
OCA_HD inline void rec_load(const T *r, T &dp, T &iD, T &s, T &yb) {
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(r);
        dp = v.x;
        iD = v.y;
        s = v.z;
        yb = v.w;
    } else {
        const double2 v0 = *reinterpret_cast<const double2 *>(r);
        const double2 v1 = *reinterpret_cast<const double2 *>(r + 2);
        dp = v0.x;
        iD = v0.y;
        s = v1.x;
        yb = v1.y;
    }
#else
    dp = r[0];
    iD = r[1];
    s = r[2];
    yb = r[3];
#endif
}
// the first two fields only (the Hessian's pass over the active faces)
template <typename T>
OCA_HD inline void rec_load2(const T *r, T &dp, T &iD) {
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(T) == 4) {
        const float2 v = *reinterpret_cast<const float2 *>(r);
        dp = v.x;
        iD = v.y;
    } else {
        const double2 v = *reinterpret_cast<const double2 *>(r);
        dp = v.x;
        iD = v.y;
    }
#else
    dp = r[0];
    iD = r[1];
#endif
}
template <typename T>
OCA_HD inline void rec_store(T *r, T dp, T iD, T s, T yb) {
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(r) = make_float4(dp, iD, s, yb);
    } else {
        *reinterpret_cast<double2 *>(r) = make_double2(dp, iD);
        *reinterpret_cast<double2 *>(r + 2) = make_double2(s, yb);
    }
#else
    r[0] = dp;
    r[1] = iD;
    r[2] = s;
    r[3] = yb;
#endif
}
template <typename T, int D>
OCA_HD inline void nrm_load(const T *p, T (&c)[D]) {
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(T) == 4 && D == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        c[0] = v.x;
        c[1] = v.y;
        return;
    } else if constexpr (sizeof(T) == 4 && D == 3) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        c[0] = v.x;
        c[1] = v.y;
        c[2] = v.z;
        return;
    } else {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        c[0] = v.x;
        c[1] = v.y;
        if constexpr (D == 3) c[2] = p[2];
    }
#else
#pragma unroll
    for (int i = 0; i < D; ++i) c[i] = p[i];
#endif
}
OCA_HD inline int low_bit(unsigned x) {
#ifdef __CUDA_ARCH__
    return __ffs(x) - 1;
#else
    return __builtin_ctz(x);
#endif
}

template <typename T, int D, int NR>
struct SsnLane {
    // robot part (per lane).  With n_k = |a_k|^2, the lambda subproblem is
    // written in its breakpoints t_k = ty_k - ta_k.u: lambda_k = bD_k max(0, t_k - tau)
    // and sum_k w_k max(0, t_k - tau) = 1 (sum b lambda = 1), where
    // Faces k >= nr are padding with ta = 0, w = bD = 0 and ty = -3e38: their
    // breakpoint never exceeds tau, so they are never active and add nothing.
    int nr;
    T ta[NR][D];  // R a_k / (prox b_k)
    T w[NR];      // b_k^2 / n_k
    T bD[NR];     // b_k / n_k
    T ty[NR];     // ybar_k n_k / b_k: the previous lambda (per pair)
    // obstacle faces (per pair): this lane's staged records and the warp's
    // world-frame normals, stride NrmStride<D>::N
    int no;
    const T *rec;
    const T *nrm;
    // slack
    T ybg;
};

template <typename T, int D, int NR>
struct SsnEval {
    T x[NR];         // max(0, t_k - tau): lambda_k = bD_k x_k
    T Kty[D + 1];
    T psi, pmag, mag;
    unsigned fmask;  // obstacle faces with mu_m > 0
    int amask;       // robot faces with lambda_k > 0
    bool gact;       // gamma > 0
};

template <typename T, int D, int NR>
OCA_HD inline void ssn_eval_staged(const SsnLane<T, D, NR> &L, T rho_p, T irho, const T bq[D + 1], const T w[D + 1],
                                   int &ahint, SsnEval<T, D, NR> &st) {
    // ahint: in, the robot faces active at the previous evaluation (or at the
    // warm start); out, those active at w
    constexpr int V = D + 1, NC = NrmStride<D>::N;
    // breakpoints t_k = ty_k - ta_k.u (prox b_k ta_k = R a_k, so ta_k.u = h_k / (prox b_k))
    T t[NR], hh[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        T hk = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) hk += L.ta[k][i] * w[1 + i];
        hh[k] = hk;
        t[k] = L.ty[k] - hk;
    }
    // threshold tau: on the active set {t_j > tau}, sum w t - tau sum w = 1.
    // The previous active set is tried first: it is the answer when its tau
    // separates it from the other breakpoints (t_k > tau exactly on the set).
    // Otherwise the full search: the active set is the largest {t_j >= t_k}
    // whose tau stays below t_k (s2 > 0, so tau_k < t_k is tested as
    // s1 - 1 < t_k s2).  One division either way.
    T bs1 = T(0), bs2 = T(0);
#pragma unroll
    for (int k = 0; k < NR; ++k)
        if ((ahint >> k) & 1) {
            bs1 += L.w[k] * t[k];
            bs2 += L.w[k];
        }
    bool hit = bs2 > T(0);
    T inv = m_rcp(hit ? bs2 : T(1));
    T tau = (bs1 - T(1)) * inv;
#pragma unroll
    for (int k = 0; k < NR; ++k)
        hit = hit && ((((ahint >> k) & 1) != 0) == (t[k] > tau));
    if (!hit) {
        bs1 = T(1);
        bs2 = T(1);
        int best_n = -1;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            T s1 = T(0), s2 = T(0);
            int n = 0;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                if (t[j] >= t[k]) {
                    s1 += L.w[j] * t[j];
                    s2 += L.w[j];
                    ++n;
                }
            }
            if (s1 - T(1) < t[k] * s2 && n > best_n) {
                best_n = n;
                bs1 = s1;
                bs2 = s2;
            }
        }
        inv = m_rcp(bs2);
        tau = (bs1 - T(1)) * inv;
    }
    // lambda_k = bD_k x_k with x_k = max(0, t_k - tau); prox n_k lambda_k^2 = prox w_k x_k^2;
    // sum lambda_k R a_k = prox sum w_k x_k ta_k
    T a1[D], rpen = T(0), rmag = T(0), mag = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) a1[i] = T(0);
    int nmask = 0;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const T xk = fmax(T(0), t[k] - tau);
        const T wx = L.w[k] * xk;
        st.x[k] = xk;
        nmask |= (xk > T(0) ? 1 : 0) << k;
        rpen += wx * xk;
        rmag += wx * (m_abs(L.ty[k]) + m_abs(hh[k]));
        mag += L.bD[k] * xk;
#pragma unroll
        for (int i = 0; i < D; ++i) a1[i] += wx * L.ta[k][i];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) a1[i] *= rho_p;
    // faces: mu_m = max(0, (s_m - h_m) iD_m); penalty mu_m (s_m - h_m) = mu_m^2 / iD_m
    // Rounding scales: a term mu r (r = s - h > 0 where mu > 0) is computed
    // from s and h with |h| <= s + r, so sum mu (s + |h|) <= 2 sum mu s + fpen
    // bounds the magnitudes that enter psi; sum mu (|d'| + 1) those of the
    // face part of K^T y (unit-scale normals).
    T fpen = T(0), fms = T(0), sd = T(0), sc[D];
#pragma unroll
    for (int i = 0; i < D; ++i) sc[i] = T(0);
    unsigned fmask = 0u;
    for (int m = 0; m < L.no; ++m) {
        T dp, iDm, s, yb, c[D];
        rec_load<T>(L.rec + 4 * m, dp, iDm, s, yb);
        nrm_load<T, D>(L.nrm + NC * m, c);
        T cw = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) cw += c[i] * w[1 + i];
        const T r = s - (w[0] * dp + cw);
        T mu = r * iDm;
        fmask |= (mu > T(0) ? 1u : 0u) << m;
        mu = fmax(mu, T(0));
        fpen += mu * r;
        fms += mu * s;
        mag += mu * (m_abs(dp) + T(1));
        sd += mu * dp;
#pragma unroll
        for (int i = 0; i < D; ++i) sc[i] += mu * c[i];
    }
    const T gam = fmax(T(0), L.ybg - w[0] * irho);
    st.Kty[0] = sd + gam;
#pragma unroll
    for (int i = 0; i < D; ++i) st.Kty[1 + i] = a1[i] + sc[i];
    T ww = T(0), bw = T(0);
#pragma unroll
    for (int i = 0; i < V; ++i) {
        ww += w[i] * w[i];
        bw += bq[i] * w[i];
    }
    const T gp = rho_p * gam * gam;
    st.psi = T(0.5) * ww - bw + T(0.5) * (fpen + gp) + rho_p * (T(0.5) * rpen + tau);
    st.pmag = T(0.5) * ww + m_abs(bw) + fms + fpen + T(0.5) * gp + rho_p * (rmag + T(2) * (m_abs(tau) + inv));
    st.mag = mag + gam;
    st.fmask = fmask;
    st.amask = nmask;
    st.gact = gam > T(0);
    ahint = nmask;
}

// H = prox I + sum_{mu_m > 0} K_m K_m^T / |K_m|^2 + e0 e0^T [gamma > 0]
//     + (lambda block on u: sum_S a a^T/n - (sum_S b a/n)(...)^T / sum_S b^2/n
//        = prox^2 (sum_S w ta ta^T - (sum_S w ta)(sum_S w ta)^T / sum_S w)),
// over the sets of the evaluation st (world frame)
template <typename T, int D, int NR>
OCA_HD inline void ssn_hess_staged(const SsnLane<T, D, NR> &L, T rho_p, const SsnEval<T, D, NR> &st,
                                   T H[D + 1][D + 1]) {
    constexpr int V = D + 1, NC = NrmStride<D>::N;
    T M[V][V];
#pragma unroll
    for (int i = 0; i < V; ++i)
#pragma unroll
        for (int j = 0; j < V; ++j) M[i][j] = T(0);
    for (unsigned fm = st.fmask; fm != 0u; fm &= fm - 1u) {
        const int m = low_bit(fm);
        T e[V], iDm;
        rec_load2<T>(L.rec + 4 * m, e[0], iDm);
        T c[D];
        nrm_load<T, D>(L.nrm + NC * m, c);
#pragma unroll
        for (int i = 0; i < D; ++i) e[1 + i] = c[i];
        T we[V];
#pragma unroll
        for (int i = 0; i < V; ++i) we[i] = iDm * e[i];
#pragma unroll
        for (int i = 0; i < V; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) M[i][j] += we[i] * e[j];
    }
    T Ha[D][D], ba[D], bb = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        ba[i] = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) Ha[i][j] = T(0);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        if ((st.amask >> k) & 1) {
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const T ai = L.w[k] * L.ta[k][i];
                ba[i] += ai;
#pragma unroll
                for (int j = 0; j <= i; ++j) Ha[i][j] += ai * L.ta[k][j];
            }
            bb += L.w[k];
        }
    }
    const T ibb = bb > T(0) ? m_rcp(bb) : T(0);
    const T r2 = rho_p * rho_p;
#pragma unroll
    for (int i = 0; i < V; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T hv = rho_p * M[i][j] + (i == j ? rho_p : T(0));
            if (i == 0 && j == 0 && st.gact) hv += T(1);
            if (i > 0 && j > 0) hv += r2 * (Ha[i - 1][j - 1] - ba[i - 1] * ba[j - 1] * ibb);
            H[i][j] = hv;
            H[j][i] = hv;
        }
}

// The part of an evaluation the solve carries from one pass to the next:
// the accepted point's x (lambda_k = bD_k x_k, the result), psi and its
// rounding scale.
template <typename T, int NR>
struct SsnKeep {
    T x[NR];
    T psi, pmag;
};

template <typename T, int D, int NR>
OCA_HD inline int ssn_solve_staged(const SsnLane<T, D, NR> &L, T rho_p, T irho, const T bq[D + 1], T w[D + 1],
                                   SsnKeep<T, NR> &st) {
    // One loop with a single evaluation site: every pass evaluates y(w) at
    // one point -- the start point, or a trial w + t d of the line search --
    // and then stops (a full Newton step that stayed in the region of its
    // Hessian), backtracks, or accepts the trial and computes the next Newton
    // direction from that evaluation.  (The same sequence of evaluations as a
    // Newton loop with a nested line search; but the evaluation code exists
    // once, and lanes of a warp in different phases share evaluation passes.)
    constexpr int V = D + 1;
    int status = OCA_PAIR_ITER_CAP;
    T dlt[V], wt[V], tstep = T(1), gd = T(0);
    bool started = false, newton = false;
    int it = 0, ls = 0;
    // robot faces active at the last evaluation; first guess: the warm start's
    int ahint = 0;
#pragma unroll
    for (int k = 0; k < NR; ++k) ahint |= (L.ty[k] > T(0) ? 1 : 0) << k;
    // the sets at the point whose Hessian gave the current direction
    unsigned hf = 0u;
    int ha = 0;
    bool hg = false;
    for (int pass = 0; pass < 1 + 60 * 30; ++pass) {
#pragma unroll
        for (int i = 0; i < V; ++i) wt[i] = started ? w[i] + tstep * dlt[i] : w[i];
        SsnEval<T, D, NR> trial;
        ssn_eval_staged<T, D, NR>(L, rho_p, irho, bq, wt, ahint, trial);
        bool stop = false;
        if (started) {
            if (newton && tstep == T(1) && trial.fmask == hf && trial.amask == ha && trial.gact == hg) {
                // F is affine between w and the trial: the Newton point is the root
                status = OCA_PAIR_OK;
                stop = true;
            } else {
                // Armijo decrease, relaxed by the rounding level of psi; psi must
                // strictly decrease unless the predicted decrease is itself below
                // that level (a tie or a rise with a larger predicted decrease is
                // real: accepting it can cycle between two regions)
                const T slack = T(8) * m_eps<T>() * (st.pmag + trial.pmag);
                const bool ok = trial.psi <= st.psi + T(1e-4) * tstep * gd + slack &&
                                (trial.psi < st.psi || -tstep * gd <= slack);
                if (!ok && ls < 29) {
                    // backtracking on psi: psi is piecewise quadratic along the ray,
                    // so the minimiser of the quadratic through psi(0), psi'(0) = gd
                    // and psi(t) is usually exact after one rejected trial
                    const T curv = trial.psi - st.psi - tstep * gd;
                    T tn = curv > T(0) ? -gd * tstep * tstep / (T(2) * curv) : T(0.5) * tstep;
                    tstep = fmin(fmax(tn, T(0.1) * tstep), T(0.5) * tstep);
                    ++ls;
                    continue;
                }
                if (!ok) {
                    status = OCA_PAIR_OK;  // no decrease at rounding level
                    stop = true;
                }
                if (++it >= 60) stop = true;
            }
        } else {
            started = true;
        }
        // accept the trial
#pragma unroll
        for (int i = 0; i < V; ++i) w[i] = wt[i];
#pragma unroll
        for (int k = 0; k < NR; ++k) st.x[k] = trial.x[k];
        st.psi = trial.psi;
        st.pmag = trial.pmag;
        if (stop) break;
        // convergence test and the next Newton direction at w
        T F[V], fn = T(0), scale = T(1) + trial.mag;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            F[i] = w[i] - bq[i] - trial.Kty[i];
            fn = fmax(fn, m_abs(F[i]));
            scale = fmax(scale, fmax(m_abs(w[i]), m_abs(bq[i])));
        }
        if (fn <= T(16) * m_eps<T>() * scale) {
            status = OCA_PAIR_OK;
            break;
        }
        if (!(fn == fn)) {
            status = OCA_PAIR_NONFINITE;
            break;
        }
        T H[V][V];
        ssn_hess_staged<T, D, NR>(L, rho_p, trial, H);
#pragma unroll
        for (int i = 0; i < V; ++i) dlt[i] = -rho_p * F[i];
        newton = chol_solve<T, V>(H, dlt, V, T(0));
        if (!newton) {
#pragma unroll
            for (int i = 0; i < V; ++i) dlt[i] = -F[i];
        }
        gd = T(0);
#pragma unroll
        for (int i = 0; i < V; ++i) gd += F[i] * dlt[i];
        if (!(gd < T(0))) {
#pragma unroll
            for (int i = 0; i < V; ++i) dlt[i] = -F[i];
            gd = T(0);
#pragma unroll
            for (int i = 0; i < V; ++i) gd -= F[i] * F[i];
            newton = false;
        }
        hf = trial.fmask;
        ha = trial.amask;
        hg = trial.gact;
        tstep = T(1);
        ls = 0;
    }
    return status;
}

// ============================================================================
// Scale LP (Sec. III-A eqn:scale_opt) through its dual (eqn:scale_opt_dual):
//   min d'^T mu  s.t.  b^T lambda = 1,  A^T lambda + C'^T mu = 0,  lambda, mu >= 0
// by a revised two-phase simplex with Bland's rule on D+1 equality rows.
// Column ids: lambda_k -> k, mu_m -> nr + m, artificial of row i -> ART + i.
// ============================================================================
template <typename T, int D>
OCA_HD inline void lp_col(const Lane<T, D> &L, int id, int ART, T col[D + 1], T &cost) {
    if (id < L.nr) {
        col[0] = ldg(L.b + id);
#pragma unroll
        for (int i = 0; i < D; ++i) col[1 + i] = ldg(L.A + id * D + i);
        cost = T(0);
    } else if (id < ART) {
        T g[D + 1];
        gen_vec<T, D>(L, id, g);  // [d'_m; c'_m]
        col[0] = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) col[1 + i] = g[1 + i];
        cost = g[0];
    } else {
#pragma unroll
        for (int i = 0; i <= D; ++i) col[i] = (i == id - ART) ? T(1) : T(0);
        cost = T(0);
    }
}

template <typename T, int D>
OCA_HD int lp_solve(const Lane<T, D> &L, int bas[D + 1], T xB[D + 1], T &alpha) {
    constexpr int V = D + 1;
    const int ART = L.nr + L.no;
    T Bi[V][V];
#pragma unroll
    for (int i = 0; i < V; ++i) {
#pragma unroll
        for (int j = 0; j < V; ++j) Bi[i][j] = (i == j) ? T(1) : T(0);
        bas[i] = ART + i;
        xB[i] = (i == 0) ? T(1) : T(0);
    }
    const T tol = T(64) * m_eps<T>();
    int status = OCA_PAIR_OK;
    int piv = 0;
    for (int phase = 1; phase <= 2; ++phase) {
        for (;;) {
            if (++piv > 64) {
                status = OCA_PAIR_ITER_CAP;
                break;
            }
            // simplex multipliers pi = c_B^T B^-1
            T cB[V], pi[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                T col[V], c;
                lp_col<T, D>(L, bas[i], ART, col, c);
                cB[i] = (phase == 1) ? (bas[i] >= ART ? T(1) : T(0)) : (bas[i] >= ART ? T(0) : c);
            }
#pragma unroll
            for (int j = 0; j < V; ++j) {
                T acc = T(0);
#pragma unroll
                for (int i = 0; i < V; ++i) acc += cB[i] * Bi[i][j];
                pi[j] = acc;
            }
            // Bland pricing: lowest id with negative reduced cost
            int enter = -1;
            for (int id = 0; id < ART && enter < 0; ++id) {
                bool basic = false;
#pragma unroll
                for (int i = 0; i < V; ++i) basic |= (bas[i] == id);
                if (basic) continue;
                T col[V], c;
                lp_col<T, D>(L, id, ART, col, c);
                if (phase == 1) c = T(0);
                T rc = c, scale = m_abs(c);
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    rc -= pi[i] * col[i];
                    scale += m_abs(pi[i] * col[i]);
                }
                if (rc < -tol * (T(1) + scale)) enter = id;
            }
            if (enter < 0) break;
            T col[V], c, dcol[V];
            lp_col<T, D>(L, enter, ART, col, c);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < V; ++k) acc += Bi[i][k] * col[k];
                dcol[i] = acc;
            }
            int r = -1;
            T best = T(0);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                if (dcol[i] > tol) {
                    const T ratio = xB[i] / dcol[i];
                    if (r < 0 || ratio < best || (ratio == best && bas[i] < bas[r])) {
                        r = i;
                        best = ratio;
                    }
                }
            }
            if (r < 0) {
                status = OCA_PAIR_DEGENERATE;  // unbounded: impossible for a bounded part
                break;
            }
            // pivot on (r, enter)
            T pr = T(0), brow[V];
#pragma unroll
            for (int i = 0; i < V; ++i)
                if (i == r) pr = dcol[i];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                T acc = T(0);
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (i == r) acc = Bi[i][k];
                brow[k] = acc / pr;
            }
            T xr = T(0);
#pragma unroll
            for (int i = 0; i < V; ++i)
                if (i == r) xr = xB[i] / pr;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                if (i == r) {
#pragma unroll
                    for (int k = 0; k < V; ++k) Bi[i][k] = brow[k];
                    xB[i] = xr;
                    bas[i] = enter;
                } else {
#pragma unroll
                    for (int k = 0; k < V; ++k) Bi[i][k] -= dcol[i] * brow[k];
                    xB[i] = fmax(T(0), xB[i] - dcol[i] * xr);
                }
            }
        }
        if (status != OCA_PAIR_OK) break;
        if (phase == 1) {
            // drive zero-level artificials out of the basis where possible
#pragma unroll
            for (int i = 0; i < V; ++i) {
                if (bas[i] >= ART) {
                    for (int id = 0; id < ART; ++id) {
                        bool basic = false;
#pragma unroll
                        for (int k = 0; k < V; ++k) basic |= (bas[k] == id);
                        if (basic) continue;
                        T col[V], c;
                        lp_col<T, D>(L, id, ART, col, c);
                        T di = T(0);
#pragma unroll
                        for (int k = 0; k < V; ++k) di += Bi[i][k] * col[k];
                        if (m_abs(di) > T(1e3) * tol) {
                            T dcol[V];
#pragma unroll
                            for (int ii = 0; ii < V; ++ii) {
                                T acc = T(0);
#pragma unroll
                                for (int k = 0; k < V; ++k) acc += Bi[ii][k] * col[k];
                                dcol[ii] = acc;
                            }
                            T brow[V];
#pragma unroll
                            for (int k = 0; k < V; ++k) brow[k] = Bi[i][k] / di;
#pragma unroll
                            for (int ii = 0; ii < V; ++ii) {
                                if (ii == i) continue;
#pragma unroll
                                for (int k = 0; k < V; ++k) Bi[ii][k] -= dcol[ii] * brow[k];
                            }
#pragma unroll
                            for (int k = 0; k < V; ++k) Bi[i][k] = brow[k];
                            bas[i] = id;
                            break;
                        }
                    }
                }
            }
        }
    }
    // refine: solve B xB = e1 directly from the final basis
    {
        T Bm[V][V], r[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            T col[V], c;
            lp_col<T, D>(L, bas[j], ART, col, c);
#pragma unroll
            for (int i = 0; i < V; ++i) Bm[i][j] = col[i];
        }
#pragma unroll
        for (int i = 0; i < V; ++i) r[i] = (i == 0) ? T(1) : T(0);
        // Gaussian elimination with partial pivoting (static indexing)
        bool ok = true;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            int pv = k;
            T pmax = m_abs(Bm[k][k]);
#pragma unroll
            for (int i = k + 1; i < V; ++i)
                if (m_abs(Bm[i][k]) > pmax) {
                    pmax = m_abs(Bm[i][k]);
                    pv = i;
                }
            if (!(pmax > T(0))) {
                ok = false;
                break;
            }
#pragma unroll
            for (int i = k + 1; i < V; ++i) {
                if (i == pv) {
#pragma unroll
                    for (int jj = 0; jj < V; ++jj) {
                        T t = Bm[k][jj];
                        Bm[k][jj] = Bm[i][jj];
                        Bm[i][jj] = t;
                    }
                    T t = r[k];
                    r[k] = r[i];
                    r[i] = t;
                }
            }
#pragma unroll
            for (int i = k + 1; i < V; ++i) {
                const T f = Bm[i][k] / Bm[k][k];
#pragma unroll
                for (int jj = k; jj < V; ++jj) Bm[i][jj] -= f * Bm[k][jj];
                r[i] -= f * r[k];
            }
        }
        if (ok) {
#pragma unroll
            for (int i = V - 1; i >= 0; --i) {
                T acc = r[i];
#pragma unroll
                for (int jj = i + 1; jj < V; ++jj) acc -= Bm[i][jj] * r[jj];
                r[i] = acc / Bm[i][i];
            }
#pragma unroll
            for (int i = 0; i < V; ++i) xB[i] = fmax(T(0), r[i]);
        }
    }
    T obj = T(0);
#pragma unroll
    for (int i = 0; i < V; ++i) {
        T col[V], c;
        lp_col<T, D>(L, bas[i], ART, col, c);
        if (bas[i] >= L.nr && bas[i] < ART) obj += c * xB[i];
    }
    alpha = -obj;
    return status;
}


// Primal point x* of eqn:scale_opt (body frame) from the final basis of
// lp_solve: the simplex multipliers pi of the dual LP solve B^T pi = c_B
// (B the basic columns, c_B their costs) and equal (-alpha*, x*).  Returns
// false if the basis matrix is singular.
template <typename T, int D>
OCA_HD inline bool lp_primal(const Lane<T, D> &L, const int bas[D + 1], T x[D]) {
    constexpr int V = D + 1;
    const int ART = L.nr + L.no;
    T M[V][V], r[V];  // M = B^T
#pragma unroll
    for (int j = 0; j < V; ++j) {
        T col[V], c;
        lp_col<T, D>(L, bas[j], ART, col, c);
#pragma unroll
        for (int i = 0; i < V; ++i) M[j][i] = col[i];
        r[j] = bas[j] >= ART ? T(0) : c;
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
        int pv = k;
        T pmax = m_abs(M[k][k]);
#pragma unroll
        for (int i = k + 1; i < V; ++i)
            if (m_abs(M[i][k]) > pmax) {
                pmax = m_abs(M[i][k]);
                pv = i;
            }
        if (!(pmax > T(0))) return false;
#pragma unroll
        for (int i = k + 1; i < V; ++i) {
            if (i == pv) {
#pragma unroll
                for (int jj = 0; jj < V; ++jj) {
                    const T t = M[k][jj];
                    M[k][jj] = M[i][jj];
                    M[i][jj] = t;
                }
                const T t = r[k];
                r[k] = r[i];
                r[i] = t;
            }
        }
#pragma unroll
        for (int i = k + 1; i < V; ++i) {
            const T f = M[i][k] / M[k][k];
#pragma unroll
            for (int jj = k; jj < V; ++jj) M[i][jj] -= f * M[k][jj];
            r[i] -= f * r[k];
        }
    }
#pragma unroll
    for (int i = V - 1; i >= 0; --i) {
        T acc = r[i];
#pragma unroll
        for (int jj = i + 1; jj < V; ++jj) acc -= M[i][jj] * r[jj];
        r[i] = acc / M[i][i];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) x[i] = r[1 + i];
    return true;
}



}  // namespace oca
