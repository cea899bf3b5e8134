/*
 * Plain FP64 CPU oracle of the scale-based collision-avoidance ADMM of
 * "GPU-Accelerated Optimization-Based Collision Avoidance" (Wu, Wang, Zhang).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or
 * constant with the CUDA path; both read the same seeded input arrays.
 *
 * Every function follows the paper's definitions in their plain form:
 *   ora_scale_lp      Sec. III-A eqn:scale_opt, solved through its dual
 *                     (Sec. III-B eqn:scale_opt_dual) by a dense two-phase
 *                     tableau simplex with Bland's rule.
 *   ora_pair_qp       Sec. IV-C eqn:const_least_square, by the paper's route:
 *                     elimination of one lambda (eqn:const_least_square_ineq),
 *                     KKT -> LCP (eqn:kkt_conditions,
 *                     eqn:linear_complementarity_problem), Lemke's method.
 *                     Optional proximal term 0.5*prox*sum_i |K_i|^2 (y_i - ybar_i)^2
 *                     (each generator's step measured in residual space).
 *   ora_dynamics      Sec. IV-A eqn:system_eqn, s_{t+1} = s_t + dt*f_c(s,u).
 *   ora_part_pose     rho(s), R(s) of Sec. IV-A and their state derivatives.
 *   ora_riccati       the step-2 LQ subproblem (SQP: one QP per iteration,
 *                     Sec. IV-B) by the textbook backward Riccati recursion.
 *   ora_riccati_scan  the same LQ subproblem in parallel-in-time form: the
 *                     stage relations of its optimality conditions composed
 *                     associatively (pairwise, in log N rounds or right to
 *                     left), giving every stage's value function P_t, p_t.
 *   ora_admm_scenario the three ADMM steps (eqn:ADMM_dual_updates,
 *                     eqn:ADMM_state_updates, eqn:ADMM_residue_updates) and
 *                     the stopping rule of Sec. IV-B, Gauss-Seidel order.
 *   ora_cert_margin   a weak-duality lower bound on alpha* (Sec. III-B).
 *
 * Parity pins of each function live in the test suite.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_MAXF 32                 /* max faces per polytope            */
#define ORA_MAXY (2 * ORA_MAXF + 1) /* max length of y = [lambda; mu; g] */
#define ORA_MAXL (ORA_MAXY + 1)     /* max LCP size                      */
#define ORA_MAXS 12                 /* max state dimension               */
#define ORA_MAXU 4                  /* max control dimension             */

enum { ORA_OK = 0, ORA_ITER_CAP = 1, ORA_FAIL = 2, ORA_BAD_INPUT = 3 };

/* ------------------------------------------------------------------------ */
/* small dense helpers                                                       */
/* ------------------------------------------------------------------------ */

/* Solve A x = b (n x n, row-major, copied) by Gaussian elimination with
 * partial pivoting.  Returns 0 on success, -1 if singular. */
static int ora_gauss_solve(int n, const double *A_in, const double *b_in, double *x) {
    double A[ORA_MAXL * ORA_MAXL], b[ORA_MAXL];
    memcpy(A, A_in, sizeof(double) * n * n);
    memcpy(b, b_in, sizeof(double) * n);
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
        if (fabs(A[piv * n + k]) < 1e-300) return -1;
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double f = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
        x[i] = s / A[i * n + i];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Scale LP, Sec. III-A eqn:scale_opt                                        */
/*   min alpha  s.t.  A x <= alpha b,  C x <= d      (body frame of part)   */
/* solved through the dual eqn:scale_opt_dual in minimisation form:         */
/*   min d^T mu  s.t.  b^T lambda = 1,  A^T lambda + C^T mu = 0,  >= 0       */
/* so alpha* = -min d^T mu.  The optimal simplex multipliers pi of the       */
/* equality rows give the primal point: x = pi[1..d], alpha = -pi[0].       */
/* ------------------------------------------------------------------------ */

static void ora_pivot(double *T, int rows, int cols, int r, int c) {
    double p = T[r * cols + c];
    for (int j = 0; j < cols; ++j) T[r * cols + j] /= p;
    for (int i = 0; i < rows; ++i) {
        if (i == r) continue;
        double f = T[i * cols + c];
        if (f == 0.0) continue;
        for (int j = 0; j < cols; ++j) T[i * cols + j] -= f * T[r * cols + j];
    }
}

/* One simplex phase with Bland's rule on tableau T (m constraint rows + one
 * reduced-cost row, last column = rhs).  Columns >= nenter never enter.
 * Returns 0 optimal, 1 unbounded, 2 pivot cap. */
static int ora_simplex_phase(double *T, int m, int cols, int nenter, int *basis) {
    const double eps = 1e-12;
    for (int it = 0; it < 5000; ++it) {
        int q = -1;
        for (int j = 0; j < nenter; ++j)
            if (T[m * cols + j] < -eps) { q = j; break; }     /* Bland: lowest index */
        if (q < 0) return 0;
        int r = -1;
        double best = 0.0;
        for (int i = 0; i < m; ++i) {
            double a = T[i * cols + q];
            if (a > eps) {
                double ratio = T[i * cols + cols - 1] / a;
                if (r < 0 || ratio < best - 1e-15 ||
                    (fabs(ratio - best) <= 1e-15 && basis[i] < basis[r])) {
                    r = i; best = ratio;
                }
            }
        }
        if (r < 0) return 1;
        ora_pivot(T, m + 1, cols, r, q);
        basis[r] = q;
    }
    return 2;
}

int ora_scale_lp(int d, int nr, const double *A, const double *b, int no, const double *Cb,
                 const double *db, double *alpha, double *lam, double *mu, double *x) {
    const int m = d + 1, n = nr + no, cols = n + m + 1;
    if (d < 2 || d > 3 || nr < 1 || no < 1 || nr > ORA_MAXF || no > ORA_MAXF) return ORA_BAD_INPUT;
    double T[(4 + 1) * (2 * ORA_MAXF + 4 + 1)];
    int basis[4];
    memset(T, 0, sizeof(double) * (m + 1) * cols);
    /* equality rows: row 0 is b^T lambda = 1, rows 1..d are A^T lambda + C^T mu = 0 */
    for (int k = 0; k < nr; ++k) {
        T[0 * cols + k] = b[k];
        for (int i = 0; i < d; ++i) T[(1 + i) * cols + k] = A[k * d + i];
    }
    for (int j = 0; j < no; ++j)
        for (int i = 0; i < d; ++i) T[(1 + i) * cols + nr + j] = Cb[j * d + i];
    for (int i = 0; i < m; ++i) {
        T[i * cols + n + i] = 1.0;          /* artificial of row i */
        basis[i] = n + i;
    }
    T[0 * cols + cols - 1] = 1.0;
    /* phase 1: minimise the sum of artificials */
    for (int j = 0; j < cols; ++j) {
        double s = 0.0;
        if (j < n || j == cols - 1)
            for (int i = 0; i < m; ++i) s += T[i * cols + j];
        T[m * cols + j] = (j < n) ? -s : (j == cols - 1 ? -s : 0.0);
    }
    if (ora_simplex_phase(T, m, cols, n, basis) != 0) return ORA_FAIL;
    if (fabs(T[m * cols + cols - 1]) > 1e-9) return ORA_FAIL; /* dual infeasible: cannot happen */
    /* drive zero-level artificials out of the basis */
    for (int i = 0; i < m; ++i) {
        if (basis[i] < n) continue;
        int q = -1;
        for (int j = 0; j < n; ++j)
            if (fabs(T[i * cols + j]) > 1e-9) { q = j; break; }
        if (q >= 0) { ora_pivot(T, m + 1, cols, i, q); basis[i] = q; }
    }
    /* phase 2: reduced costs of c = (0 for lambda, d' for mu) */
    for (int j = 0; j < cols; ++j) {
        double cj = (j >= nr && j < n) ? db[j - nr] : 0.0;
        if (j == cols - 1) cj = 0.0;
        double s = 0.0;
        for (int i = 0; i < m; ++i) {
            int bi = basis[i];
            double cb = (bi >= nr && bi < n) ? db[bi - nr] : 0.0;
            s += cb * T[i * cols + j];
        }
        T[m * cols + j] = cj - s;
    }
    int st = ora_simplex_phase(T, m, cols, n, basis);
    if (st != 0) return ORA_FAIL;
    double yv[2 * ORA_MAXF];
    memset(yv, 0, sizeof(double) * n);
    for (int i = 0; i < m; ++i)
        if (basis[i] < n) yv[basis[i]] = T[i * cols + cols - 1];
    double obj = 0.0;
    for (int j = 0; j < no; ++j) obj += db[j] * yv[nr + j];
    *alpha = -obj;
    if (lam) for (int k = 0; k < nr; ++k) lam[k] = yv[k];
    if (mu) for (int j = 0; j < no; ++j) mu[j] = yv[nr + j];
    if (x) {
        /* pi_i = -(reduced cost of the artificial column of row i) */
        for (int i = 0; i < d; ++i) x[i] = -T[m * cols + n + 1 + i];
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Pair QP, Sec. IV-C eqn:const_least_square                                 */
/*   min 0.5|K^T y + bq|^2 (+ 0.5 prox |y - ybar|^2)                        */
/*   s.t. kappa^T y = 1 (kappa = [b; 0; 0]),  y >= 0,                       */
/* y = [lambda (nr); mu (no); gamma], rows of K (body frame of the part):   */
/*   lambda_k : [0, a_k^T],  mu_m : [d'_m, c'_m^T],  gamma : [1, 0].        */
/* Route: eliminate y_e (e = largest b_e, lowest index on ties) with        */
/* kappa_e^T y_e = eta - kappa_u^T y_u, giving eqn:const_least_square_ineq,  */
/* then the KKT conditions as the LCP w = M z + q, z = [y_u; phi], solved by  */
/* Lemke's complementary pivoting (covering vector of ones, lexicographic    */
/* minimum-ratio rule).                                                     */
/* ------------------------------------------------------------------------ */

/* Lemke's method for w = M z + q, w,z >= 0, w^T z = 0.  n <= ORA_MAXL.
 * Degenerate LCPs (many optimal y of the pair QP) make floating-point
 * pivoting fragile, so the pivots are chosen on q + delta, with delta a
 * fixed generic perturbation of relative size 1e-9 (a numerical stand-in for
 * the symbolic lexicographic perturbation), and the solution is then
 * recomputed exactly from the final complementary basis with the original q:
 * x_B = B^{-1} q, B^{-1} being the w-columns of the tableau.
 * Returns 0 solved, 1 ray termination, 2 pivot cap. */
static int ora_lemke(int n, const double *M, const double *q_in, double *z, int *npiv) {
    const int cols = 2 * n + 2;          /* w(n) | z(n) | z0 | rhs */
    const int cz0 = 2 * n, crhs = 2 * n + 1;
    static __thread double T[ORA_MAXL * (2 * ORA_MAXL + 2)];
    int basis[ORA_MAXL];
    const double eps = 1e-13;
    double q[ORA_MAXL], qmax = 0.0;
    *npiv = 0;
    int neg = 0;
    for (int i = 0; i < n; ++i) {
        if (q_in[i] < 0.0) neg = 1;
        qmax = fmax(qmax, fabs(q_in[i]));
    }
    for (int i = 0; i < n; ++i) z[i] = 0.0;
    if (!neg) return 0;
    for (int i = 0; i < n; ++i) {
        const double frac = fmod(0.6180339887498949 * (i + 1), 1.0);
        q[i] = q_in[i] + 1e-9 * (1.0 + qmax) * (0.5 + frac);
    }
    memset(T, 0, sizeof(double) * n * cols);
    for (int i = 0; i < n; ++i) {
        T[i * cols + i] = 1.0;
        for (int j = 0; j < n; ++j) T[i * cols + n + j] = -M[i * n + j];
        T[i * cols + cz0] = -1.0;
        T[i * cols + crhs] = q[i];
        basis[i] = i;
    }
    /* initial pivot: z0 enters, the row of the most negative q_i leaves
     * (largest index among ties keeps the tableau lexicographically positive) */
    int r = 0;
    for (int i = 1; i < n; ++i) if (q[i] <= q[r]) r = i;
    int leaving = basis[r];
    ora_pivot(T, n, cols, r, cz0);
    basis[r] = cz0;
    *npiv = 1;
    for (int it = 0; it < 50 * n + 50; ++it) {
        int enter = (leaving < n) ? leaving + n : leaving - n;   /* complement */
        /* lexicographic minimum-ratio test: minimum ratio over rows with a
         * positive entry, then filter the tie set column by column of B^{-1}
         * (the w columns), preferring z0 when it is tied */
        double cmax = 0.0;
        for (int i = 0; i < n; ++i) cmax = fmax(cmax, fabs(T[i * cols + enter]));
        const double atol = eps * (1.0 + cmax);
        double th = INFINITY;
        for (int i = 0; i < n; ++i) {
            double a = T[i * cols + enter];
            if (a > atol) th = fmin(th, T[i * cols + crhs] / a);
        }
        int rr = -1;
        if (th < INFINITY) {
            int cand[ORA_MAXL], nc = 0;
            const double ttol = 1e-12 * (1.0 + fabs(th));
            for (int i = 0; i < n; ++i) {
                double a = T[i * cols + enter];
                if (a > atol && T[i * cols + crhs] / a <= th + ttol) cand[nc++] = i;
            }
            for (int c = 0; c < nc; ++c)
                if (basis[cand[c]] == cz0) rr = cand[c];
            for (int k = 0; rr < 0 && k < n && nc > 1; ++k) {
                double mn = INFINITY;
                for (int c = 0; c < nc; ++c) mn = fmin(mn, T[cand[c] * cols + k] / T[cand[c] * cols + enter]);
                const double ktol = 1e-12 * (1.0 + fabs(mn));
                int m2 = 0;
                for (int c = 0; c < nc; ++c)
                    if (T[cand[c] * cols + k] / T[cand[c] * cols + enter] <= mn + ktol) cand[m2++] = cand[c];
                nc = m2;
            }
            if (rr < 0) rr = cand[0];
        }
        if (rr < 0) return 1;
        leaving = basis[rr];
        ora_pivot(T, n, cols, rr, enter);
        basis[rr] = enter;
        ++*npiv;
        if (leaving == cz0) {
            /* exact resolve with the unperturbed q on the final basis */
            int ok = 1;
            double xb[ORA_MAXL];
            for (int i = 0; i < n; ++i) {
                double acc = 0.0;
                for (int k = 0; k < n; ++k) acc += T[i * cols + k] * q_in[k];
                xb[i] = acc;
                if (acc < -1e-9 * (1.0 + qmax)) ok = 0;
            }
            for (int i = 0; i < n; ++i)
                if (basis[i] >= n && basis[i] < 2 * n)
                    z[basis[i] - n] = ok ? fmax(0.0, xb[i]) : T[i * cols + crhs];
            return 0;
        }
    }
    return 2;
}

int ora_pair_qp(int d, int nr, const double *A, const double *b, int no, const double *Cb,
                const double *db, const double *bq, double prox, const double *ybar, double *y,
                double *v, double *obj, int *npiv_out) {
    const int V = d + 1, ny = nr + no + 1;
    if (d < 2 || d > 3 || nr < 1 || no < 0 || nr > ORA_MAXF || no > ORA_MAXF) return ORA_BAD_INPUT;
    double K[ORA_MAXY * 4], kappa[ORA_MAXY];
    memset(K, 0, sizeof(K));
    memset(kappa, 0, sizeof(kappa));
    for (int k = 0; k < nr; ++k) {
        for (int i = 0; i < d; ++i) K[k * V + 1 + i] = A[k * d + i];
        kappa[k] = b[k];
    }
    for (int m = 0; m < no; ++m) {
        K[(nr + m) * V] = db[m];
        for (int i = 0; i < d; ++i) K[(nr + m) * V + 1 + i] = Cb[m * d + i];
    }
    K[(nr + no) * V] = 1.0;
    const double eta = 1.0;
    int e = 0;
    for (int k = 1; k < nr; ++k) if (b[k] > b[e]) e = k;
    /* index map of the remaining components y_u */
    int uidx[ORA_MAXY];
    int n = 0;
    for (int i = 0; i < ny; ++i) if (i != e) uidx[n++] = i;
    double Kt[ORA_MAXY * 4], kt[ORA_MAXY], bt[4];
    const double ke = kappa[e];
    for (int a = 0; a < n; ++a) {
        int i = uidx[a];
        kt[a] = kappa[i] / ke;                                /* kappa~ = kappa_u kappa_e^-1 */
        for (int c = 0; c < V; ++c) Kt[a * V + c] = K[i * V + c] - kt[a] * K[e * V + c];
    }
    for (int c = 0; c < V; ++c) bt[c] = bq[c] + K[e * V + c] * eta / ke;  /* b~ */
    const double etat = eta / ke;                                     /* eta~ */
    /* LCP of size n+1: M = [[H, kt], [-kt^T, 0]], q = [f; eta~].
     * The proximal term is measured in residual space:
     * 0.5 prox sum_i |K_i|^2 (y_i - ybar_i)^2 = 0.5 prox (y - ybar)^T Dg (y - ybar),
     * which with y = y_0 + N y_u adds prox N^T Dg N to H and
     * prox N^T Dg (y_0 - ybar) to f. */
    double Dg[ORA_MAXY];
    for (int i = 0; i < ny; ++i) {
        double s2 = 0.0;
        for (int c = 0; c < V; ++c) s2 += K[i * V + c] * K[i * V + c];
        Dg[i] = s2;
    }
    const int L = n + 1;
    double M[ORA_MAXL * ORA_MAXL], q[ORA_MAXL], z[ORA_MAXL];
    for (int a = 0; a < n; ++a) {
        for (int c2 = 0; c2 < n; ++c2) {
            double s = 0.0;
            for (int c = 0; c < V; ++c) s += Kt[a * V + c] * Kt[c2 * V + c];
            if (prox > 0.0) s += prox * ((a == c2 ? Dg[uidx[a]] : 0.0) + Dg[e] * kt[a] * kt[c2]);
            M[a * L + c2] = s;
        }
        M[a * L + n] = kt[a];
        M[n * L + a] = -kt[a];
        double f = 0.0;
        for (int c = 0; c < V; ++c) f += Kt[a * V + c] * bt[c];
        if (prox > 0.0) {
            double yb_e = ybar ? ybar[e] : 0.0, yb_a = ybar ? ybar[uidx[a]] : 0.0;
            f += prox * (-Dg[e] * kt[a] * (etat - yb_e) - Dg[uidx[a]] * yb_a);
        }
        q[a] = f;
    }
    M[n * L + n] = 0.0;
    q[n] = etat;
    int npiv = 0;
    int st = ora_lemke(L, M, q, z, &npiv);
    if (npiv_out) *npiv_out = npiv;
    double yy[ORA_MAXY];
    double s = 0.0;
    for (int a = 0; a < n; ++a) { yy[uidx[a]] = z[a]; s += kt[a] * z[a]; }
    yy[e] = etat - s;                                      /* y_e = kappa_e^-T (eta - kappa_u^T y_u) */
    for (int i = 0; i < ny; ++i) y[i] = yy[i];
    double o = 0.0;
    for (int c = 0; c < V; ++c) {
        double vc = bq[c];
        for (int i = 0; i < ny; ++i) vc += K[i * V + c] * yy[i];
        if (v) v[c] = vc;
        o += 0.5 * vc * vc;
    }
    if (obj) *obj = o;
    if (st == 1) return ORA_FAIL;
    if (st == 2) return ORA_ITER_CAP;
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Models: eqn:system_eqn with s_{t+1} = s_t + dt * f_c(s_t, u_t)            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int kind;          /* 0 bicycle (4,2), 1 trailer (5,2), 2 quad (12,4) */
    double dt;
    double param[8];
    double Qs[ORA_MAXS], Qu[ORA_MAXU];
    double s_lo[ORA_MAXS], s_hi[ORA_MAXS];  /* state boxes of eqn:MPC_opt_origin (+-1e30: none) */
    double u_lo[ORA_MAXU], u_hi[ORA_MAXU];  /* control boxes */
} ora_model;

static int ora_ns(int kind) { return kind == 0 ? 4 : kind == 1 ? 5 : 12; }
static int ora_nu(int kind) { return kind == 2 ? 4 : 2; }
static int ora_dim(int kind) { return kind == 2 ? 3 : 2; }

static void ora_rot3(double phi, double th, double psi, double R[9], double dR[3][9]) {
    double cf = cos(phi), sf = sin(phi), ct = cos(th), st = sin(th), cp = cos(psi), sp = sin(psi);
    double Rx[9] = {1, 0, 0, 0, cf, -sf, 0, sf, cf}, dRx[9] = {0, 0, 0, 0, -sf, -cf, 0, cf, -sf};
    double Ry[9] = {ct, 0, st, 0, 1, 0, -st, 0, ct}, dRy[9] = {-st, 0, ct, 0, 0, 0, -ct, 0, -st};
    double Rz[9] = {cp, -sp, 0, sp, cp, 0, 0, 0, 1}, dRz[9] = {-sp, -cp, 0, cp, -sp, 0, 0, 0, 0};
    /* R = Rz Ry Rx (ZYX Euler: yaw, pitch, roll) */
    const double *F[3][3] = {{Rz, Ry, dRx}, {Rz, dRy, Rx}, {dRz, Ry, Rx}};
    for (int w = 0; w < 4; ++w) {
        const double *a = (w == 3) ? Rz : F[w][0];
        const double *bb = (w == 3) ? Ry : F[w][1];
        const double *c = (w == 3) ? Rx : F[w][2];
        double t[9], out[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int k = 0; k < 3; ++k) s += a[i * 3 + k] * bb[k * 3 + j];
                t[i * 3 + j] = s;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int k = 0; k < 3; ++k) s += t[i * 3 + k] * c[k * 3 + j];
                out[i * 3 + j] = s;
            }
        if (w == 3) memcpy(R, out, sizeof(out));
        else if (dR) memcpy(dR[w], out, sizeof(out));
    }
}

/* Continuous-time f_c(s,u) and its Jacobians fs = df/ds (ns x ns),
 * fu = df/du (ns x nu); any output may be NULL. */
void ora_dynamics(const ora_model *md, const double *s, const double *u, double *f, double *fs,
                  double *fu) {
    const int ns = ora_ns(md->kind), nu = ora_nu(md->kind);
    double F[ORA_MAXS], Fs[ORA_MAXS * ORA_MAXS], Fu[ORA_MAXS * ORA_MAXU];
    memset(F, 0, sizeof(F));
    memset(Fs, 0, sizeof(Fs));
    memset(Fu, 0, sizeof(Fu));
    if (md->kind == 0 || md->kind == 1) {
        /* kinematic bicycle with the steering entered as path curvature
         * kappa = tan(delta) / L:  x' = v cos th, y' = v sin th, th' = v kappa, v' = a */
        double th = s[2], v = s[3], a = u[0], kap = u[1];
        F[0] = v * cos(th);
        F[1] = v * sin(th);
        F[2] = v * kap;
        F[3] = a;
        Fs[0 * ns + 2] = -v * sin(th); Fs[0 * ns + 3] = cos(th);
        Fs[1 * ns + 2] = v * cos(th);  Fs[1 * ns + 3] = sin(th);
        Fs[2 * ns + 3] = kap;
        Fu[2 * nu + 1] = v;
        Fu[3 * nu + 0] = 1.0;
        if (md->kind == 1) {
            /* off-axle hitch M behind the rear axle, trailer axle L2 behind the hitch:
             * psi' = (v/L2) sin(th-psi) - (v M kappa / L2) cos(th-psi) */
            const double Mh = md->param[1], L2 = md->param[2];
            double ps = s[4], sd = sin(th - ps), cd = cos(th - ps);
            F[4] = v / L2 * sd - v * Mh * kap / L2 * cd;
            double dth = v / L2 * cd + v * Mh * kap / L2 * sd;
            Fs[4 * ns + 2] = dth;
            Fs[4 * ns + 4] = -dth;
            Fs[4 * ns + 3] = sd / L2 - Mh * kap / L2 * cd;
            Fu[4 * nu + 1] = -v * Mh / L2 * cd;
        }
    } else {
        const double m = md->param[0], g = md->param[1];
        const double Jx = md->param[2], Jy = md->param[3], Jz = md->param[4];
        const double ell = md->param[5], km = md->param[6];
        double phi = s[6], th = s[7], psi = s[8], p = s[9], q = s[10], r = s[11];
        double R[9], dR[3][9];
        ora_rot3(phi, th, psi, R, dR);
        double thrust = m * g;                       /* hover total */
        for (int i = 0; i < 4; ++i) thrust += u[i];
        /* p_dot = v */
        for (int i = 0; i < 3; ++i) { F[i] = s[3 + i]; Fs[i * ns + 3 + i] = 1.0; }
        /* v_dot = R e3 * T / m - g e3 */
        for (int i = 0; i < 3; ++i) {
            F[3 + i] = R[i * 3 + 2] * thrust / m - (i == 2 ? g : 0.0);
            for (int a = 0; a < 3; ++a) Fs[(3 + i) * ns + 6 + a] = dR[a][i * 3 + 2] * thrust / m;
            for (int k = 0; k < 4; ++k) Fu[(3 + i) * nu + k] = R[i * 3 + 2] / m;
        }
        /* eta_dot = W(eta) omega (ZYX Euler kinematics) */
        double cf = cos(phi), sf = sin(phi), ct = cos(th), tt = tan(th), sc = 1.0 / ct;
        F[6] = p + sf * tt * q + cf * tt * r;
        F[7] = cf * q - sf * r;
        F[8] = sf * sc * q + cf * sc * r;
        double sec2 = sc * sc;
        Fs[6 * ns + 6] = cf * tt * q - sf * tt * r;
        Fs[6 * ns + 7] = sf * sec2 * q + cf * sec2 * r;
        Fs[6 * ns + 9] = 1.0; Fs[6 * ns + 10] = sf * tt; Fs[6 * ns + 11] = cf * tt;
        Fs[7 * ns + 6] = -sf * q - cf * r;
        Fs[7 * ns + 10] = cf; Fs[7 * ns + 11] = -sf;
        Fs[8 * ns + 6] = cf * sc * q - sf * sc * r;
        Fs[8 * ns + 7] = (sf * q + cf * r) * sc * tt;
        Fs[8 * ns + 10] = sf * sc; Fs[8 * ns + 11] = cf * sc;
        /* omega_dot = J^-1 (tau - omega x J omega); "+" layout: rotors 1..4 on +x,+y,-x,-y */
        F[9] = (ell * (u[1] - u[3]) - q * r * (Jz - Jy)) / Jx;
        F[10] = (ell * (u[2] - u[0]) - p * r * (Jx - Jz)) / Jy;
        F[11] = (km * (u[0] - u[1] + u[2] - u[3]) - p * q * (Jy - Jx)) / Jz;
        Fs[9 * ns + 10] = -r * (Jz - Jy) / Jx; Fs[9 * ns + 11] = -q * (Jz - Jy) / Jx;
        Fs[10 * ns + 9] = -r * (Jx - Jz) / Jy; Fs[10 * ns + 11] = -p * (Jx - Jz) / Jy;
        Fs[11 * ns + 9] = -q * (Jy - Jx) / Jz; Fs[11 * ns + 10] = -p * (Jy - Jx) / Jz;
        Fu[9 * nu + 1] = ell / Jx; Fu[9 * nu + 3] = -ell / Jx;
        Fu[10 * nu + 2] = ell / Jy; Fu[10 * nu + 0] = -ell / Jy;
        Fu[11 * nu + 0] = km / Jz; Fu[11 * nu + 1] = -km / Jz;
        Fu[11 * nu + 2] = km / Jz; Fu[11 * nu + 3] = -km / Jz;
    }
    if (f) memcpy(f, F, sizeof(double) * ns);
    if (fs) memcpy(fs, Fs, sizeof(double) * ns * ns);
    if (fu) memcpy(fu, Fu, sizeof(double) * ns * nu);
}

/* Pose of a robot part (Sec. IV-A: y = R(s) x + rho(s)).
 * link 0: vehicle body (2D: rear axle (x,y), heading theta; 3D: position, ZYX Euler).
 * link 1: trailer (2D): hitch M behind the rear axle, heading psi = s[4].
 * off: part centre in its link frame.  Outputs: rho (d), R (d x d row-major),
 * drho (d x ns), dR (ns x d x d); derivative outputs may be NULL. */
void ora_part_pose(const ora_model *md, int link, const double *off, const double *s,
                   double *rho, double *R, double *drho, double *dR) {
    const int ns = ora_ns(md->kind), d = ora_dim(md->kind);
    double Dr[3 * ORA_MAXS], DR[ORA_MAXS * 9];
    memset(Dr, 0, sizeof(Dr));
    memset(DR, 0, sizeof(DR));
    if (d == 2) {
        int ai = (link == 1) ? 4 : 2;                   /* state index of the part heading */
        double a = s[ai], c = cos(a), sn = sin(a);
        R[0] = c; R[1] = -sn; R[2] = sn; R[3] = c;
        double Rp[4] = {-sn, -c, c, -sn};
        rho[0] = s[0] + c * off[0] - sn * off[1];
        rho[1] = s[1] + sn * off[0] + c * off[1];
        Dr[0 * ns + 0] = 1.0; Dr[1 * ns + 1] = 1.0;
        Dr[0 * ns + ai] += Rp[0] * off[0] + Rp[1] * off[1];
        Dr[1 * ns + ai] += Rp[2] * off[0] + Rp[3] * off[1];
        if (link == 1) {
            double th = s[2], ct = cos(th), st = sin(th), Mh = md->param[1];
            rho[0] += -Mh * ct;
            rho[1] += -Mh * st;
            Dr[0 * ns + 2] += Mh * st;
            Dr[1 * ns + 2] += -Mh * ct;
        }
        for (int k = 0; k < 4; ++k) DR[ai * 4 + k] = Rp[k];
    } else {
        double dR3[3][9];
        ora_rot3(s[6], s[7], s[8], R, dR3);
        for (int i = 0; i < 3; ++i) {
            double t = 0;
            for (int k = 0; k < 3; ++k) t += R[i * 3 + k] * off[k];
            rho[i] = s[i] + t;
            Dr[i * ns + i] = 1.0;
            for (int a = 0; a < 3; ++a) {
                double tt = 0;
                for (int k = 0; k < 3; ++k) tt += dR3[a][i * 3 + k] * off[k];
                Dr[i * ns + 6 + a] = tt;
            }
        }
        for (int a = 0; a < 3; ++a) memcpy(&DR[(6 + a) * 9], dR3[a], sizeof(double) * 9);
    }
    if (drho) memcpy(drho, Dr, sizeof(double) * d * ns);
    if (dR) memcpy(dR, DR, sizeof(double) * ns * d * d);
}

/* ------------------------------------------------------------------------ */
/* Step 2 LQ subproblem by backward Riccati recursion (FP64).               */
/*   min sum_{t=0}^{N} 0.5 s_t^T Q_t s_t + q_t^T s_t                         */
/*     + sum_{t=0}^{N-1} 0.5 u_t^T R_t u_t + r_t^T u_t                       */
/*   s.t. s_{t+1} = A_t s_t + B_t u_t + c_t,  s_0 given.                     */
/* ------------------------------------------------------------------------ */
int ora_riccati(int ns, int nu, int N, const double *A, const double *B, const double *c,
                const double *Q, const double *q, const double *R, const double *r,
                const double *s0, double *s, double *u) {
    double *Kg = (double *)malloc(sizeof(double) * N * nu * ns);
    double *kg = (double *)malloc(sizeof(double) * N * nu);
    double P[ORA_MAXS * ORA_MAXS], p[ORA_MAXS];
    memcpy(P, Q + (size_t)N * ns * ns, sizeof(double) * ns * ns);
    memcpy(p, q + (size_t)N * ns, sizeof(double) * ns);
    int ok = 0;
    for (int t = N - 1; t >= 0; --t) {
        const double *At = A + (size_t)t * ns * ns, *Bt = B + (size_t)t * ns * nu;
        const double *ct = c + (size_t)t * ns;
        double PA[ORA_MAXS * ORA_MAXS], PB[ORA_MAXS * ORA_MAXU], w[ORA_MAXS];
        for (int i = 0; i < ns; ++i) {
            for (int j = 0; j < ns; ++j) {
                double acc = 0;
                for (int k = 0; k < ns; ++k) acc += P[i * ns + k] * At[k * ns + j];
                PA[i * ns + j] = acc;
            }
            for (int j = 0; j < nu; ++j) {
                double acc = 0;
                for (int k = 0; k < ns; ++k) acc += P[i * ns + k] * Bt[k * nu + j];
                PB[i * nu + j] = acc;
            }
            double acc = p[i];
            for (int k = 0; k < ns; ++k) acc += P[i * ns + k] * ct[k];
            w[i] = acc;                                    /* P c + p */
        }
        double Quu[ORA_MAXU * ORA_MAXU], Qus[ORA_MAXU * ORA_MAXS], qu[ORA_MAXU];
        for (int i = 0; i < nu; ++i) {
            for (int j = 0; j < nu; ++j) {
                double acc = R[(size_t)t * nu * nu + i * nu + j];
                for (int k = 0; k < ns; ++k) acc += Bt[k * nu + i] * PB[k * nu + j];
                Quu[i * nu + j] = acc;
            }
            for (int j = 0; j < ns; ++j) {
                double acc = 0;
                for (int k = 0; k < ns; ++k) acc += Bt[k * nu + i] * PA[k * ns + j];
                Qus[i * ns + j] = acc;
            }
            double acc = r[(size_t)t * nu + i];
            for (int k = 0; k < ns; ++k) acc += Bt[k * nu + i] * w[k];
            qu[i] = acc;
        }
        double Qss[ORA_MAXS * ORA_MAXS], qs[ORA_MAXS];
        for (int i = 0; i < ns; ++i) {
            for (int j = 0; j < ns; ++j) {
                double acc = Q[(size_t)t * ns * ns + i * ns + j];
                for (int k = 0; k < ns; ++k) acc += At[k * ns + i] * PA[k * ns + j];
                Qss[i * ns + j] = acc;
            }
            double acc = q[(size_t)t * ns + i];
            for (int k = 0; k < ns; ++k) acc += At[k * ns + i] * w[k];
            qs[i] = acc;
        }
        /* K = -Quu^-1 Qus, k = -Quu^-1 qu */
        double *Kt = Kg + (size_t)t * nu * ns, *kt = kg + (size_t)t * nu;
        for (int j = 0; j < ns; ++j) {
            double rhs[ORA_MAXU], sol[ORA_MAXU];
            for (int i = 0; i < nu; ++i) rhs[i] = -Qus[i * ns + j];
            if (ora_gauss_solve(nu, Quu, rhs, sol)) { ok = -1; break; }
            for (int i = 0; i < nu; ++i) Kt[i * ns + j] = sol[i];
        }
        {
            double rhs[ORA_MAXU];
            for (int i = 0; i < nu; ++i) rhs[i] = -qu[i];
            if (ora_gauss_solve(nu, Quu, rhs, kt)) ok = -1;
        }
        if (ok) break;
        for (int i = 0; i < ns; ++i) {
            for (int j = 0; j < ns; ++j) {
                double acc = Qss[i * ns + j];
                for (int k = 0; k < nu; ++k) acc += Qus[k * ns + i] * Kt[k * ns + j];
                P[i * ns + j] = acc;
            }
            double acc = qs[i];
            for (int k = 0; k < nu; ++k) acc += Qus[k * ns + i] * kt[k];
            p[i] = acc;
        }
        /* symmetrise */
        for (int i = 0; i < ns; ++i)
            for (int j = i + 1; j < ns; ++j) {
                double m = 0.5 * (P[i * ns + j] + P[j * ns + i]);
                P[i * ns + j] = P[j * ns + i] = m;
            }
    }
    if (!ok) {
        memcpy(s, s0, sizeof(double) * ns);
        for (int t = 0; t < N; ++t) {
            const double *Kt = Kg + (size_t)t * nu * ns, *kt = kg + (size_t)t * nu;
            double *st = s + (size_t)t * ns, *ut = u + (size_t)t * nu, *sn = s + (size_t)(t + 1) * ns;
            for (int i = 0; i < nu; ++i) {
                double acc = kt[i];
                for (int k = 0; k < ns; ++k) acc += Kt[i * ns + k] * st[k];
                ut[i] = acc;
            }
            const double *At = A + (size_t)t * ns * ns, *Bt = B + (size_t)t * ns * nu;
            for (int i = 0; i < ns; ++i) {
                double acc = c[(size_t)t * ns + i];
                for (int k = 0; k < ns; ++k) acc += At[i * ns + k] * st[k];
                for (int k = 0; k < nu; ++k) acc += Bt[i * nu + k] * ut[k];
                sn[i] = acc;
            }
        }
    }
    free(Kg);
    free(kg);
    return ok ? ORA_FAIL : ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 2 in parallel-in-time form (the same LQ problem as ora_riccati).    */
/* Its optimality conditions, with costate lam_t = dV_t/ds_t and the        */
/* stationarity u_t = -R_t^-1 (B_t^T lam_{t+1} + r_t), link each stage's     */
/* state and costate linearly:                                              */
/*   s_{t+1} = A_t s_t + b_t - C_t lam_{t+1},                                */
/*   lam_t   = J_t s_t - eta_t + A_t^T lam_{t+1},                            */
/* with b_t = c_t - B_t R_t^-1 r_t, C_t = B_t R_t^-1 B_t^T, J_t = Q_t,         */
/* eta_t = -q_t; the terminal condition lam_N = Q_N s_N + q_N is the         */
/* element (A, b, C, J, eta) = (0, 0, 0, Q_N, -q_N).  Two consecutive        */
/* relations (1: i -> j, then 2: j -> k) give, on eliminating s_j and lam_j, */
/* one of the same form, with M = (I + C1 J2)^-1 (invertible: C1, J2 are     */
/* positive semidefinite) and M^T = (I + J2 C1)^-1:                         */
/*   A = A2 M A1,  b = A2 M (b1 + C1 eta2) + b2,  C = A2 M C1 A2^T + C2,      */
/*   J = J1 + A1^T M^T J2 A1,  eta = eta1 + A1^T M^T (eta2 - J2 b1).          */
/* Elimination is order-free, so the composition is associative: the       */
/* suffix e_t o ... o e_N, whose A is 0, states lam_t = J s_t - eta, i.e.    */
/* the value function's P_t = J, p_t = -eta.  tree != 0 forms every suffix  */
/* in ceil(log2(N+1)) rounds of pairwise compositions (element t takes      */
/* element t + 2^r); tree == 0 forms them right to left.  The solution then */
/* follows by the forward rollout u_t = -(R + B^T P B)^-1 (B^T (P (A s + c)   */
/* + p) + r), s_{t+1} = A s + B u + c with P, p of stage t+1.                 */
/* P_out [N+1][ns][ns], p_out [N+1][ns] may be NULL.                        */
/* ------------------------------------------------------------------------ */
static int ora_lq_compose(int n, const double *e1, const double *e2, double *e) {
    /* element layout: A [n*n], b [n], C [n*n], J [n*n], eta [n] */
    const int nn = n * n;
    const double *A1 = e1, *b1 = e1 + nn, *C1 = b1 + n, *J1 = C1 + nn, *h1 = J1 + nn;
    const double *A2 = e2, *b2 = e2 + nn, *C2 = b2 + n, *J2 = C2 + nn, *h2 = J2 + nn;
    double *A = e, *b = e + nn, *C = b + n, *J = C + nn, *h = J + nn;
    double T[ORA_MAXS * ORA_MAXS], Tt[ORA_MAXS * ORA_MAXS];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = (i == j) ? 1.0 : 0.0, acct = acc;
            for (int k = 0; k < n; ++k) {
                acc += C1[i * n + k] * J2[k * n + j];   /* I + C1 J2 */
                acct += J2[i * n + k] * C1[k * n + j];  /* I + J2 C1 */
            }
            T[i * n + j] = acc;
            Tt[i * n + j] = acct;
        }
    /* X = M [A1 | b1 + C1 eta2 | C1 A2^T], column by column */
    double XA[ORA_MAXS * ORA_MAXS], Xb[ORA_MAXS], XC[ORA_MAXS * ORA_MAXS], col[ORA_MAXS], sol[ORA_MAXS];
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) col[i] = A1[i * n + j];
        if (ora_gauss_solve(n, T, col, sol)) return -1;
        for (int i = 0; i < n; ++i) XA[i * n + j] = sol[i];
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += C1[i * n + k] * A2[j * n + k];  /* (C1 A2^T)[i][j] */
            col[i] = acc;
        }
        if (ora_gauss_solve(n, T, col, sol)) return -1;
        for (int i = 0; i < n; ++i) XC[i * n + j] = sol[i];
    }
    for (int i = 0; i < n; ++i) {
        double acc = b1[i];
        for (int k = 0; k < n; ++k) acc += C1[i * n + k] * h2[k];
        col[i] = acc;
    }
    if (ora_gauss_solve(n, T, col, Xb)) return -1;
    /* Y = M^T [J2 A1 | eta2 - J2 b1] */
    double YJ[ORA_MAXS * ORA_MAXS], Ye[ORA_MAXS];
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += J2[i * n + k] * A1[k * n + j];
            col[i] = acc;
        }
        if (ora_gauss_solve(n, Tt, col, sol)) return -1;
        for (int i = 0; i < n; ++i) YJ[i * n + j] = sol[i];
    }
    for (int i = 0; i < n; ++i) {
        double acc = h2[i];
        for (int k = 0; k < n; ++k) acc -= J2[i * n + k] * b1[k];
        col[i] = acc;
    }
    if (ora_gauss_solve(n, Tt, col, Ye)) return -1;
    for (int i = 0; i < n; ++i) {
        double ab = b2[i], ah = h1[i];
        for (int k = 0; k < n; ++k) {
            ab += A2[i * n + k] * Xb[k];
            ah += A1[k * n + i] * Ye[k];
        }
        b[i] = ab;
        h[i] = ah;
        for (int j = 0; j < n; ++j) {
            double aa = 0.0, ac = C2[i * n + j], aj = J1[i * n + j];
            for (int k = 0; k < n; ++k) {
                aa += A2[i * n + k] * XA[k * n + j];
                ac += A2[i * n + k] * XC[k * n + j];
                aj += A1[k * n + i] * YJ[k * n + j];
            }
            A[i * n + j] = aa;
            C[i * n + j] = ac;
            J[i * n + j] = aj;
        }
    }
    return 0;
}

int ora_riccati_scan(int ns, int nu, int N, const double *A, const double *B, const double *c,
                     const double *Q, const double *q, const double *R, const double *r,
                     const double *s0, double *s, double *u, double *P_out, double *p_out, int tree) {
    if (ns < 1 || ns > ORA_MAXS || nu < 1 || nu > ORA_MAXU || N < 0) return ORA_BAD_INPUT;
    const int n = ns, nn = ns * ns, es = 3 * nn + 2 * ns, E = N + 1;
    double *cur = (double *)malloc(sizeof(double) * (size_t)es * E);
    double *nxt = (double *)malloc(sizeof(double) * (size_t)es * E);
    int ok = (cur && nxt) ? 0 : -1;
    /* the stage elements */
    for (int t = 0; t < E && ok == 0; ++t) {
        double *e = cur + (size_t)t * es;
        double *Ae = e, *be = e + nn, *Ce = be + n, *Je = Ce + nn, *he = Je + nn;
        memcpy(Je, Q + (size_t)t * nn, sizeof(double) * nn);
        for (int i = 0; i < n; ++i) he[i] = -q[(size_t)t * n + i];
        if (t == N) {
            memset(Ae, 0, sizeof(double) * nn);
            memset(be, 0, sizeof(double) * n);
            memset(Ce, 0, sizeof(double) * nn);
            continue;
        }
        const double *At = A + (size_t)t * nn, *Bt = B + (size_t)t * n * nu, *Rt = R + (size_t)t * nu * nu;
        memcpy(Ae, At, sizeof(double) * nn);
        /* W = R^-1 B^T (nu x n), z = R^-1 r */
        double W[ORA_MAXU * ORA_MAXS], z[ORA_MAXU], rhs[ORA_MAXU], sol[ORA_MAXU];
        for (int j = 0; j < n; ++j) {
            for (int a = 0; a < nu; ++a) rhs[a] = Bt[j * nu + a];
            if (ora_gauss_solve(nu, Rt, rhs, sol)) { ok = -1; break; }
            for (int a = 0; a < nu; ++a) W[a * n + j] = sol[a];
        }
        if (ok != 0 || ora_gauss_solve(nu, Rt, r + (size_t)t * nu, z)) { ok = -1; break; }
        for (int i = 0; i < n; ++i) {
            double acc = c[(size_t)t * n + i];
            for (int a = 0; a < nu; ++a) acc -= Bt[i * nu + a] * z[a];
            be[i] = acc;
            for (int j = 0; j < n; ++j) {
                double cc = 0.0;
                for (int a = 0; a < nu; ++a) cc += Bt[i * nu + a] * W[a * n + j];
                Ce[i * n + j] = cc;
            }
        }
    }
    /* suffix compositions */
    if (ok == 0 && tree) {
        for (int d = 1; d < E && ok == 0; d *= 2) {
            for (int t = 0; t < E && ok == 0; ++t) {
                if (t + d < E) ok = ora_lq_compose(n, cur + (size_t)t * es, cur + (size_t)(t + d) * es,
                                                   nxt + (size_t)t * es);
                else memcpy(nxt + (size_t)t * es, cur + (size_t)t * es, sizeof(double) * es);
            }
            double *sw = cur; cur = nxt; nxt = sw;
        }
    } else if (ok == 0) {
        for (int t = E - 2; t >= 0 && ok == 0; --t) {
            ok = ora_lq_compose(n, cur + (size_t)t * es, cur + (size_t)(t + 1) * es, nxt);
            memcpy(cur + (size_t)t * es, nxt, sizeof(double) * es);
        }
    }
    /* value functions and the forward rollout */
    if (ok == 0) {
        if (P_out || p_out)
            for (int t = 0; t < E; ++t) {
                const double *e = cur + (size_t)t * es;
                if (P_out) memcpy(P_out + (size_t)t * nn, e + 2 * nn + n, sizeof(double) * nn);
                if (p_out)
                    for (int i = 0; i < n; ++i) p_out[(size_t)t * n + i] = -e[3 * nn + n + i];
            }
        memcpy(s, s0, sizeof(double) * n);
        for (int t = 0; t < N && ok == 0; ++t) {
            const double *e = cur + (size_t)(t + 1) * es;
            const double *P = e + 2 * nn + n, *mh = e + 3 * nn + n;  /* P_{t+1}; -p_{t+1} */
            const double *At = A + (size_t)t * nn, *Bt = B + (size_t)t * n * nu, *ct = c + (size_t)t * n;
            const double *x = s + (size_t)t * n;
            double y[ORA_MAXS], w[ORA_MAXS], PB[ORA_MAXS * ORA_MAXU];
            for (int i = 0; i < n; ++i) {
                double acc = ct[i];
                for (int k = 0; k < n; ++k) acc += At[i * n + k] * x[k];
                y[i] = acc;                                   /* A s + c */
            }
            for (int i = 0; i < n; ++i) {
                double acc = -mh[i];
                for (int k = 0; k < n; ++k) acc += P[i * n + k] * y[k];
                w[i] = acc;                                   /* P (A s + c) + p */
                for (int a = 0; a < nu; ++a) {
                    double pb = 0.0;
                    for (int k = 0; k < n; ++k) pb += P[i * n + k] * Bt[k * nu + a];
                    PB[i * nu + a] = pb;
                }
            }
            double Quu[ORA_MAXU * ORA_MAXU], rhs[ORA_MAXU];
            for (int a = 0; a < nu; ++a) {
                double acc = r[(size_t)t * nu + a];
                for (int k = 0; k < n; ++k) acc += Bt[k * nu + a] * w[k];
                rhs[a] = -acc;
                for (int b2 = 0; b2 < nu; ++b2) {
                    double qq = R[(size_t)t * nu * nu + a * nu + b2];
                    for (int k = 0; k < n; ++k) qq += Bt[k * nu + a] * PB[k * nu + b2];
                    Quu[a * nu + b2] = qq;
                }
            }
            double *ut = u + (size_t)t * nu;
            if (ora_gauss_solve(nu, Quu, rhs, ut)) { ok = -1; break; }
            double *xn = s + (size_t)(t + 1) * n;
            for (int i = 0; i < n; ++i) {
                double acc = y[i];
                for (int a = 0; a < nu; ++a) acc += Bt[i * nu + a] * ut[a];
                xn[i] = acc;
            }
        }
    }
    free(cur);
    free(nxt);
    return ok == 0 ? ORA_OK : ORA_FAIL;
}

/* ------------------------------------------------------------------------ */
/* Scene description (same arrays as the C-ABI, double precision)           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dim, n_scen, fo_max, fr_max;
    const int *obs_begin, *obs_nf;
    const double *obs_C, *obs_d;            /* [M][FO][dim], [M][FO] */
    const int *part_begin, *part_nf, *part_link;
    const double *part_A, *part_b, *part_off;
    const int *horizon;
} ora_scene;

typedef struct {
    double sigma, eps_pri, eps_dual, prox;
    int max_iter;
    int jacobi;        /* 1: literal superscript-k (Jacobi) reading of steps 2 and 3 */
    double rho_box;    /* penalty of the box-constraint block (state/control bounds); 0: off */
    double damp;       /* proximal weight 0.5*damp*|(s,u) - (s,u)^k|^2 in step 2      */
} ora_admm_params;

/* Transform obstacle j into the body frame of a part with pose (rho, R):
 * C' = C R (rows R^T c_m),  d' = d - C rho. */
static void ora_obstacle_body(int d, int no, const double *C, const double *dd, const double *rho,
                              const double *R, double *Cb, double *db) {
    for (int m = 0; m < no; ++m) {
        double cr = 0;
        for (int i = 0; i < d; ++i) cr += C[m * d + i] * rho[i];
        db[m] = dd[m] - cr;
        for (int i = 0; i < d; ++i) {
            double acc = 0;
            for (int k = 0; k < d; ++k) acc += R[k * d + i] * C[m * d + k];
            Cb[m * d + i] = acc;
        }
    }
}

/* The per-pair ADMM residuals of Sec. IV-A:
 *   T = 1 + (d - C rho)^T mu + gamma,   R = A^T lambda + (C R)^T mu.   */
static void ora_pair_residual(int d, int nr, const double *A, int no, const double *C,
                              const double *dd, const double *rho, const double *Rm,
                              const double *y, int fr_max, int fo_max, double *T, double *Rv) {
    const double *lam = y, *mu = y + fr_max, gam = y[fr_max + fo_max];
    double t = 1.0 + gam;
    for (int m = 0; m < no; ++m) {
        double cr = 0;
        for (int i = 0; i < d; ++i) cr += C[m * d + i] * rho[i];
        t += (dd[m] - cr) * mu[m];
    }
    *T = t;
    for (int i = 0; i < d; ++i) {
        double acc = 0;
        for (int k = 0; k < nr; ++k) acc += A[k * d + i] * lam[k];
        for (int m = 0; m < no; ++m) {
            double cri = 0;                                  /* (C R)_{m,i} */
            for (int k = 0; k < d; ++k) cri += C[m * d + k] * Rm[k * d + i];
            acc += cri * mu[m];
        }
        Rv[i] = acc;
    }
}

/* Gauss-Newton terms of one pair residual r(s_t) = [T + zeta; R + xi]
 * (Sec. IV-A T and R, linearised in s_t at fixed y as step 2 needs):
 *   r0 = r(s_t),  J = dr/ds_t ((d+1) x ns),
 *   dT/ds = -(C^T mu)^T drho/ds,   dR/ds_a = (C dR/ds_a)^T mu.           */
void ora_pair_gn(const ora_model *md, int d, int nr, const double *A, int no, const double *C,
                 const double *dd, const double *rho, const double *R, const double *drho,
                 const double *dR, const double *y, int fr_max, int fo_max, double zeta,
                 const double *xi, double *r0, double *J) {
    const int ns = ora_ns(md->kind);
    const double *mu = y + fr_max;
    double T, Rv[3];
    ora_pair_residual(d, nr, A, no, C, dd, rho, R, y, fr_max, fo_max, &T, Rv);
    r0[0] = T + zeta;
    for (int i = 0; i < d; ++i) r0[1 + i] = Rv[i] + xi[i];
    double Cmu[3] = {0, 0, 0};
    for (int mm = 0; mm < no; ++mm)
        for (int i = 0; i < d; ++i) Cmu[i] += C[mm * d + i] * mu[mm];
    for (int a = 0; a < ns; ++a) {
        double acc = 0;
        for (int i = 0; i < d; ++i) acc -= Cmu[i] * drho[i * ns + a];
        J[0 * ns + a] = acc;
        for (int i = 0; i < d; ++i) {
            double v2 = 0;
            for (int k = 0; k < d; ++k) v2 += dR[a * d * d + k * d + i] * Cmu[k];
            J[(1 + i) * ns + a] = v2;
        }
    }
}

/* One scenario of the ADMM (Sec. IV-B), Gauss-Seidel order:
 *   step 1 (eqn:ADMM_dual_updates): y^{k+1} = pair QP at (s^k, zeta^k, xi^k)
 *   step 2 (eqn:ADMM_state_updates): one LQ (SQP) step at (s^k, u^k) with
 *          y^{k+1}: linearised dynamics, Gauss-Newton linearisation of each
 *          pair residual r = [T + zeta; R + xi] in s_t, Riccati solve
 *   step 3 (eqn:ADMM_residue_updates): zeta += T(s^{k+1}, y^{k+1}),
 *          xi += R(s^{k+1}, y^{k+1})
 *   stop when sum(dzeta^2 + |dxi|^2) <= eps_pri and
 *             sum(|dlambda|^2 + |dmu|^2) <= eps_dual.
 * Arrays of the scenario (pair-major y [P][ny_max], zeta [P], xi [P][d],
 * s [(N+1)][ns], u [N][ns]) are updated in place.
 * out[0] = iterations, out[1] = r_pri, out[2] = r_dual, out[3] = cost F. */
int ora_admm_scenario(const ora_model *md, const ora_scene *sc, int scen, const ora_admm_params *pr,
                      const double *s_ref, double *s, double *u, double *y, double *zeta,
                      double *xi, double *out) {
    const int d = sc->dim, ns = ora_ns(md->kind), nu = ora_nu(md->kind);
    const int N = sc->horizon[scen];
    const int m0 = sc->obs_begin[scen], M = sc->obs_begin[scen + 1] - m0;
    const int p0 = sc->part_begin[scen], NP = sc->part_begin[scen + 1] - p0;
    const int FO = sc->fo_max, FR = sc->fr_max, NY = FR + FO + 1;
    const size_t P = (size_t)M * NP * N;
    int status = ORA_ITER_CAP, it = 0;
    double rp = 0, rd = 0;
    double *ynew = (double *)malloc(sizeof(double) * P * NY);
    double *Aq = (double *)calloc((size_t)N * ns * ns, sizeof(double));
    double *Bq = (double *)calloc((size_t)N * ns * nu, sizeof(double));
    double *cq = (double *)calloc((size_t)N * ns, sizeof(double));
    double *Qq = (double *)calloc((size_t)(N + 1) * ns * ns, sizeof(double));
    double *qq = (double *)calloc((size_t)(N + 1) * ns, sizeof(double));
    double *Rq = (double *)calloc((size_t)N * nu * nu, sizeof(double));
    double *rq = (double *)calloc((size_t)N * nu, sizeof(double));
    double *sn = (double *)malloc(sizeof(double) * (N + 1) * ns);
    double *un = (double *)malloc(sizeof(double) * N * nu);
    /* box block: bounded copies z and scaled duals w of the states and controls */
    double *zs = (double *)malloc(sizeof(double) * (N + 1) * ns), *ws = (double *)calloc((size_t)(N + 1) * ns, sizeof(double));
    double *zu = (double *)malloc(sizeof(double) * N * nu), *wu = (double *)calloc((size_t)N * nu, sizeof(double));
    for (int t = 0; t <= N; ++t)
        for (int i = 0; i < ns; ++i)
            zs[(size_t)t * ns + i] = fmin(fmax(s[(size_t)t * ns + i], md->s_lo[i]), md->s_hi[i]);
    for (int t = 0; t < N; ++t)
        for (int i = 0; i < nu; ++i)
            zu[(size_t)t * nu + i] = fmin(fmax(u[(size_t)t * nu + i], md->u_lo[i]), md->u_hi[i]);
    for (it = 0; it < pr->max_iter; ++it) {
        /* ---- step 1: pair QPs at s^k ---- */
        rd = 0.0;
        int qp_fail = 0;
        for (int j = 0; j < M; ++j) {
            const int gm = m0 + j, no = sc->obs_nf[gm];
            const double *C = sc->obs_C + (size_t)gm * FO * d, *dd = sc->obs_d + (size_t)gm * FO;
            for (int pt = 0; pt < NP; ++pt) {
                const int gp = p0 + pt, nr = sc->part_nf[gp];
                const double *A = sc->part_A + (size_t)gp * FR * d, *b = sc->part_b + (size_t)gp * FR;
                for (int t = 1; t <= N; ++t) {
                    const size_t p = ((size_t)j * NP + pt) * N + (t - 1);
                    double rho[3], R[9], Cb[ORA_MAXF * 3], db[ORA_MAXF];
                    ora_part_pose(md, sc->part_link[gp], sc->part_off + (size_t)gp * d,
                                  s + (size_t)t * ns, rho, R, NULL, NULL);
                    ora_obstacle_body(d, no, C, dd, rho, R, Cb, db);
                    double bq[4], yy[ORA_MAXY], yb[ORA_MAXY];
                    bq[0] = 1.0 + zeta[p];
                    for (int i = 0; i < d; ++i) bq[1 + i] = xi[p * d + i];
                    /* compact ybar = [lambda (nr); mu (no); gamma] */
                    const double *yo = y + p * NY;
                    for (int k = 0; k < nr; ++k) yb[k] = yo[k];
                    for (int mm = 0; mm < no; ++mm) yb[nr + mm] = yo[FR + mm];
                    yb[nr + no] = yo[FR + FO];
                    int st = ora_pair_qp(d, nr, A, b, no, Cb, db, bq, pr->prox, yb, yy, NULL, NULL, NULL);
                    if (st != ORA_OK) qp_fail = 1;
                    double *yn = ynew + p * NY;
                    memset(yn, 0, sizeof(double) * NY);
                    for (int k = 0; k < nr; ++k) yn[k] = yy[k];
                    for (int mm = 0; mm < no; ++mm) yn[FR + mm] = yy[nr + mm];
                    yn[FR + FO] = yy[nr + no];
                    for (int k = 0; k < FR + FO; ++k) {          /* lambda and mu only */
                        double dlt = yn[k] - yo[k];
                        rd += dlt * dlt;
                    }
                }
            }
        }
        (void)qp_fail;
        /* ---- step 2: one LQ step (y^{k+1}, zeta^k, xi^k) ---- */
        const double *yq = pr->jacobi ? y : ynew;
        for (int t = 0; t < N; ++t) {
            double f[ORA_MAXS], fs[ORA_MAXS * ORA_MAXS], fu[ORA_MAXS * ORA_MAXU];
            const double *st = s + (size_t)t * ns, *ut = u + (size_t)t * nu;
            ora_dynamics(md, st, ut, f, fs, fu);
            for (int i = 0; i < ns; ++i) {
                double acc = st[i] + md->dt * f[i];
                for (int k = 0; k < ns; ++k) {
                    double a = (i == k ? 1.0 : 0.0) + md->dt * fs[i * ns + k];
                    Aq[(size_t)t * ns * ns + i * ns + k] = a;
                    acc -= a * st[k];
                }
                for (int k = 0; k < nu; ++k) {
                    double bb = md->dt * fu[i * nu + k];
                    Bq[(size_t)t * ns * nu + i * nu + k] = bb;
                    acc -= bb * ut[k];
                }
                cq[(size_t)t * ns + i] = acc;
            }
            for (int i = 0; i < nu; ++i) {
                for (int k = 0; k < nu; ++k) Rq[(size_t)t * nu * nu + i * nu + k] = (i == k) ? 2.0 * md->Qu[i] : 0.0;
                rq[(size_t)t * nu + i] = 0.0;
                /* proximal damping and the box block's augmented term */
                Rq[(size_t)t * nu * nu + i * nu + i] += pr->damp;
                rq[(size_t)t * nu + i] -= pr->damp * ut[i];
                if (md->u_lo[i] > -1e29 || md->u_hi[i] < 1e29) {
                    Rq[(size_t)t * nu * nu + i * nu + i] += pr->rho_box;
                    rq[(size_t)t * nu + i] -= pr->rho_box * (zu[(size_t)t * nu + i] - wu[(size_t)t * nu + i]);
                }
            }
        }
        for (int t = 0; t <= N; ++t) {
            double *Qt = Qq + (size_t)t * ns * ns, *qt = qq + (size_t)t * ns;
            const double *sr = s_ref + (size_t)t * ns;
            for (int i = 0; i < ns; ++i) {
                for (int k = 0; k < ns; ++k) Qt[i * ns + k] = (i == k) ? 2.0 * md->Qs[i] : 0.0;
                qt[i] = -2.0 * md->Qs[i] * sr[i];
                if (t >= 1) {
                    Qt[i * ns + i] += pr->damp;
                    qt[i] -= pr->damp * s[(size_t)t * ns + i];
                    if (md->s_lo[i] > -1e29 || md->s_hi[i] < 1e29) {
                        Qt[i * ns + i] += pr->rho_box;
                        qt[i] -= pr->rho_box * (zs[(size_t)t * ns + i] - ws[(size_t)t * ns + i]);
                    }
                }
            }
        }
        for (int t = 1; t <= N; ++t) {
            /* Gauss-Newton terms sigma J^T J and sigma J^T r0 of every pair at step t */
            double H[ORA_MAXS * ORA_MAXS], g[ORA_MAXS];
            memset(H, 0, sizeof(H));
            memset(g, 0, sizeof(g));
            const double *sb = s + (size_t)t * ns;
            for (int pt = 0; pt < NP; ++pt) {
                const int gp = p0 + pt, nr = sc->part_nf[gp];
                const double *A = sc->part_A + (size_t)gp * FR * d;
                double rho[3], R[9], drho[3 * ORA_MAXS], dR[ORA_MAXS * 9];
                ora_part_pose(md, sc->part_link[gp], sc->part_off + (size_t)gp * d, sb, rho, R, drho, dR);
                for (int j = 0; j < M; ++j) {
                    const int gm = m0 + j, no = sc->obs_nf[gm];
                    const double *C = sc->obs_C + (size_t)gm * FO * d, *dd = sc->obs_d + (size_t)gm * FO;
                    const size_t p = ((size_t)j * NP + pt) * N + (t - 1);
                    const double *yp = yq + p * NY;
                    double r0[4], J[4 * ORA_MAXS];
                    ora_pair_gn(md, d, nr, A, no, C, dd, rho, R, drho, dR, yp, FR, FO, zeta[p],
                                xi + p * d, r0, J);
                    for (int a = 0; a < ns; ++a) {
                        for (int bidx = 0; bidx < ns; ++bidx) {
                            double acc = 0;
                            for (int r = 0; r <= d; ++r) acc += J[r * ns + a] * J[r * ns + bidx];
                            H[a * ns + bidx] += pr->sigma * acc;
                        }
                        double acc = 0;
                        for (int r = 0; r <= d; ++r) acc += J[r * ns + a] * r0[r];
                        g[a] += pr->sigma * acc;
                    }
                }
            }
            double *Qt = Qq + (size_t)t * ns * ns, *qt = qq + (size_t)t * ns;
            for (int a = 0; a < ns; ++a) {
                double hs = 0;
                for (int bidx = 0; bidx < ns; ++bidx) {
                    Qt[a * ns + bidx] += H[a * ns + bidx];
                    hs += H[a * ns + bidx] * sb[bidx];
                }
                qt[a] += g[a] - hs;                 /* linear term of 0.5|r0 + J (s - sbar)|^2 */
            }
        }
        int finite = 1;
        if (ora_riccati(ns, nu, N, Aq, Bq, cq, Qq, qq, Rq, rq, s, sn, un) == ORA_OK) {
            for (int k = 0; k < (N + 1) * ns; ++k) finite &= isfinite(sn[k]) != 0;
            for (int k = 0; k < N * nu; ++k) finite &= isfinite(un[k]) != 0;
        } else {
            finite = 0;
        }
        if (!finite) {  /* singular or non-finite trajectory step: the iteration has diverged */
            status = ORA_FAIL;
            break;
        }
        /* ---- box block: z = clip((s,u)^{k+1} + w), w += (s,u)^{k+1} - z ---- */
        double rpb = 0.0, rdb = 0.0;
        for (int t = 1; t <= N && pr->rho_box > 0.0; ++t)
            for (int i = 0; i < ns; ++i) {
                if (!(md->s_lo[i] > -1e29 || md->s_hi[i] < 1e29)) continue;
                const size_t k2 = (size_t)t * ns + i;
                const double zn = fmin(fmax(sn[k2] + ws[k2], md->s_lo[i]), md->s_hi[i]);
                rdb += (zn - zs[k2]) * (zn - zs[k2]);
                zs[k2] = zn;
                ws[k2] += sn[k2] - zn;
                rpb += (sn[k2] - zn) * (sn[k2] - zn);
            }
        for (int t = 0; t < N && pr->rho_box > 0.0; ++t)
            for (int i = 0; i < nu; ++i) {
                if (!(md->u_lo[i] > -1e29 || md->u_hi[i] < 1e29)) continue;
                const size_t k2 = (size_t)t * nu + i;
                const double zn = fmin(fmax(un[k2] + wu[k2], md->u_lo[i]), md->u_hi[i]);
                rdb += (zn - zu[k2]) * (zn - zu[k2]);
                zu[k2] = zn;
                wu[k2] += un[k2] - zn;
                rpb += (un[k2] - zn) * (un[k2] - zn);
            }
        /* ---- step 3: zeta += T(s^{k+1}, y^{k+1}), xi += R(s^{k+1}, y^{k+1}) ---- */
        const double *s3 = pr->jacobi ? s : sn;
        rp = rpb;
        rd += rdb;
        for (int j = 0; j < M; ++j) {
            const int gm = m0 + j, no = sc->obs_nf[gm];
            const double *C = sc->obs_C + (size_t)gm * FO * d, *dd = sc->obs_d + (size_t)gm * FO;
            for (int pt = 0; pt < NP; ++pt) {
                const int gp = p0 + pt, nr = sc->part_nf[gp];
                const double *A = sc->part_A + (size_t)gp * FR * d;
                for (int t = 1; t <= N; ++t) {
                    const size_t p = ((size_t)j * NP + pt) * N + (t - 1);
                    double rho[3], R[9], T, Rv[3];
                    ora_part_pose(md, sc->part_link[gp], sc->part_off + (size_t)gp * d,
                                  s3 + (size_t)t * ns, rho, R, NULL, NULL);
                    ora_pair_residual(d, nr, A, no, C, dd, rho, R, (pr->jacobi ? y : ynew) + p * NY,
                                      FR, FO, &T, Rv);
                    zeta[p] += T;
                    rp += T * T;
                    for (int i = 0; i < d; ++i) { xi[p * d + i] += Rv[i]; rp += Rv[i] * Rv[i]; }
                }
            }
        }
        memcpy(y, ynew, sizeof(double) * P * NY);
        memcpy(s, sn, sizeof(double) * (N + 1) * ns);
        memcpy(u, un, sizeof(double) * N * nu);
        if (rp <= pr->eps_pri && rd <= pr->eps_dual) { status = ORA_OK; ++it; break; }
    }
    double F = 0;
    for (int t = 0; t <= N; ++t)
        for (int i = 0; i < ns; ++i) {
            double e = s[(size_t)t * ns + i] - s_ref[(size_t)t * ns + i];
            F += md->Qs[i] * e * e;
        }
    for (int t = 0; t < N; ++t)
        for (int i = 0; i < nu; ++i) F += md->Qu[i] * u[(size_t)t * nu + i] * u[(size_t)t * nu + i];
    out[0] = it;
    out[1] = rp;
    out[2] = rd;
    out[3] = F;
    free(ynew); free(Aq); free(Bq); free(cq); free(Qq); free(qq); free(Rq); free(rq);
    free(sn); free(un); free(zs); free(ws); free(zu); free(wu);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Weak-duality certificate margin (Sec. III-B).  For lambda, mu >= 0 and    */
/* any primal-feasible (alpha, x):  lambda^T(Ax - alpha b) + mu^T(C'x - d')  */
/* <= 0, so alpha b^T lambda >= r^T x - d'^T mu with r = A^T lambda + C'^T mu.*/
/* With |x| <= alpha D (x lies in alpha P, D = max vertex norm of P):        */
/*   alpha* >= -d'^T mu / (b^T lambda + |r| D).                              */
/* ------------------------------------------------------------------------ */
double ora_cert_margin(int d, int nr, const double *A, const double *b, int no, const double *Cb,
                       const double *db, const double *lam, const double *mu) {
    /* D: max norm over the vertices of {A x <= b}, by enumerating d-subsets of faces */
    double D = 0.0;
    int idx[3];
    for (idx[0] = 0; idx[0] < nr; ++idx[0])
        for (idx[1] = idx[0] + 1; idx[1] < nr; ++idx[1])
            for (idx[2] = (d == 3 ? idx[1] + 1 : 0); idx[2] < (d == 3 ? nr : 1); ++idx[2]) {
                double Mx[9], rhs[3], xx[3];
                for (int a = 0; a < d; ++a) {
                    for (int i = 0; i < d; ++i) Mx[a * d + i] = A[idx[a] * d + i];
                    rhs[a] = b[idx[a]];
                }
                if (ora_gauss_solve(d, Mx, rhs, xx)) continue;
                int feas = 1;
                for (int k = 0; k < nr && feas; ++k) {
                    double s = 0;
                    for (int i = 0; i < d; ++i) s += A[k * d + i] * xx[i];
                    if (s > b[k] + 1e-9 * (1.0 + fabs(b[k]))) feas = 0;
                }
                if (!feas) continue;
                double nn = 0;
                for (int i = 0; i < d; ++i) nn += xx[i] * xx[i];
                if (sqrt(nn) > D) D = sqrt(nn);
            }
    double bl = 0, dm = 0, rr = 0;
    for (int k = 0; k < nr; ++k) bl += b[k] * lam[k];
    for (int m = 0; m < no; ++m) dm += db[m] * mu[m];
    for (int i = 0; i < d; ++i) {
        double r = 0;
        for (int k = 0; k < nr; ++k) r += A[k * d + i] * lam[k];
        for (int m = 0; m < no; ++m) r += Cb[m * d + i] * mu[m];
        rr += r * r;
    }
    double den = bl + sqrt(rr) * D;
    return den > 0 ? -dm / den : -INFINITY;
}

/* ------------------------------------------------------------------------ */
/* Batch drivers over a whole scene (OpenMP over scenarios / pairs).         */
/* ------------------------------------------------------------------------ */

static void ora_pair_decode(const ora_scene *sc, const long long *pair_begin, long long p, int *scen,
                            int *j, int *pt, int *t) {
    int lo = 0, hi = sc->n_scen - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (pair_begin[mid] <= p) lo = mid; else hi = mid - 1;
    }
    *scen = lo;
    long long r = p - pair_begin[lo];
    int N = sc->horizon[lo], NP = sc->part_begin[lo + 1] - sc->part_begin[lo];
    *t = (int)(r % N) + 1;
    r /= N;
    *pt = (int)(r % NP);
    *j = (int)(r / NP);
}

/* For each listed pair: alpha*, lambda*, mu* (pair-major, padded to FR / FO),
 * primal x* (body frame) and the certificate margin.  states: [sum(N+1)][ns]. */
int ora_scale_batch(const ora_model *md, const ora_scene *sc, const long long *pair_begin,
                    const long long *state_begin, const double *states, long long n_list,
                    const long long *plist, double *alpha, double *lam, double *mu, double *x,
                    double *margin, int *status, int nthreads) {
    const int d = sc->dim, ns = ora_ns(md->kind), FO = sc->fo_max, FR = sc->fr_max;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (long long l = 0; l < n_list; ++l) {
        int scen, j, pt, t;
        ora_pair_decode(sc, pair_begin, plist[l], &scen, &j, &pt, &t);
        const int gm = sc->obs_begin[scen] + j, gp = sc->part_begin[scen] + pt;
        const int no = sc->obs_nf[gm], nr = sc->part_nf[gp];
        double rho[3], R[9], Cb[ORA_MAXF * 3], db[ORA_MAXF], la[ORA_MAXF], m2[ORA_MAXF], xx[3], al;
        ora_part_pose(md, sc->part_link[gp], sc->part_off + (size_t)gp * d,
                      states + (size_t)(state_begin[scen] + t) * ns, rho, R, NULL, NULL);
        ora_obstacle_body(d, no, sc->obs_C + (size_t)gm * FO * d, sc->obs_d + (size_t)gm * FO, rho, R, Cb, db);
        const double *A = sc->part_A + (size_t)gp * FR * d, *b = sc->part_b + (size_t)gp * FR;
        int st = ora_scale_lp(d, nr, A, b, no, Cb, db, &al, la, m2, xx);
        alpha[l] = al;
        if (lam) { for (int k = 0; k < FR; ++k) lam[l * FR + k] = k < nr ? la[k] : 0.0; }
        if (mu) { for (int k = 0; k < FO; ++k) mu[l * FO + k] = k < no ? m2[k] : 0.0; }
        if (x) for (int i = 0; i < d; ++i) x[l * d + i] = xx[i];
        if (margin) margin[l] = ora_cert_margin(d, nr, A, b, no, Cb, db, la, m2);
        if (status) status[l] = st;
    }
    return 0;
}

/* Pair QPs for the listed pairs.  zeta [P], xi [P][d], y_in/y_out [n_list][NY]
 * (pair-major, padded), v [n_list][d+1], obj [n_list]. */
int ora_pair_qp_batch(const ora_model *md, const ora_scene *sc, const long long *pair_begin,
                      const long long *state_begin, const double *states, const double *zeta,
                      const double *xi, double prox, long long n_list, const long long *plist,
                      const double *y_in, double *y_out, double *v, double *obj, int *status,
                      int nthreads) {
    const int d = sc->dim, ns = ora_ns(md->kind), FO = sc->fo_max, FR = sc->fr_max, NY = FR + FO + 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (long long l = 0; l < n_list; ++l) {
        int scen, j, pt, t;
        long long p = plist[l];
        ora_pair_decode(sc, pair_begin, p, &scen, &j, &pt, &t);
        const int gm = sc->obs_begin[scen] + j, gp = sc->part_begin[scen] + pt;
        const int no = sc->obs_nf[gm], nr = sc->part_nf[gp];
        double rho[3], R[9], Cb[ORA_MAXF * 3], db[ORA_MAXF];
        ora_part_pose(md, sc->part_link[gp], sc->part_off + (size_t)gp * d,
                      states + (size_t)(state_begin[scen] + t) * ns, rho, R, NULL, NULL);
        ora_obstacle_body(d, no, sc->obs_C + (size_t)gm * FO * d, sc->obs_d + (size_t)gm * FO, rho, R, Cb, db);
        double bq[4], yb[ORA_MAXY], yy[ORA_MAXY], vv[4], o;
        bq[0] = 1.0 + zeta[p];
        for (int i = 0; i < d; ++i) bq[1 + i] = xi[p * d + i];
        const double *yo = y_in + l * NY;
        for (int k = 0; k < nr; ++k) yb[k] = yo[k];
        for (int m = 0; m < no; ++m) yb[nr + m] = yo[FR + m];
        yb[nr + no] = yo[FR + FO];
        int st = ora_pair_qp(d, nr, sc->part_A + (size_t)gp * FR * d, sc->part_b + (size_t)gp * FR, no,
                             Cb, db, bq, prox, yb, yy, vv, &o, NULL);
        double *yn = y_out + l * NY;
        memset(yn, 0, sizeof(double) * NY);
        for (int k = 0; k < nr; ++k) yn[k] = yy[k];
        for (int m = 0; m < no; ++m) yn[FR + m] = yy[nr + m];
        yn[FR + FO] = yy[nr + no];
        if (v) for (int c = 0; c <= d; ++c) v[l * (d + 1) + c] = vv[c];
        if (obj) obj[l] = o;
        if (status) status[l] = st;
    }
    return 0;
}

/* Whole ADMM solves of the listed scenarios (OpenMP over scenarios).
 * All arrays are the full-scene arrays (pair-major y [P][NY]); only the
 * listed scenarios' slices are touched.  report [S][4] as in ora_admm_scenario. */
int ora_admm_batch(const ora_model *md, const ora_scene *sc, const ora_admm_params *pr,
                   const long long *pair_begin, const long long *state_begin, const long long *ctrl_begin,
                   const double *s_ref, double *s, double *u, double *y, double *zeta, double *xi,
                   int n_list, const int *slist, double *report, int *status, int nthreads) {
    const int d = sc->dim, ns = ora_ns(md->kind), nu = ora_nu(md->kind);
    const int NY = sc->fr_max + sc->fo_max + 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int l = 0; l < n_list; ++l) {
        int scen = slist[l];
        long long pb = pair_begin[scen], sb = state_begin[scen], cb = ctrl_begin[scen];
        status[scen] = ora_admm_scenario(md, sc, scen, pr, s_ref + sb * ns, s + sb * ns, u + cb * nu,
                                         y + pb * NY, zeta + pb, xi + pb * d, report + (size_t)scen * 4);
    }
    return 0;
}

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
