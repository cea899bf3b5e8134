// Host build of the pair kernel's staged Newton solve (oca_solvers.cuh,
// compiled for the CPU: no GPU is needed) against the unstaged body-frame
// solve of the same proximal pair QP (Sec. IV-C eqn:const_least_square with
// the proximal term), on seeded random pairs.  Prints one line per case:
//   <name> <pairs> <max relative |y_staged - y_unstaged|> <pairs not OK>
// The staged solve is set up as the kernel stages it: robot faces in their
// breakpoint form, each obstacle face as a record [d', iD, s, ybar], normals
// in the warp-buffer stride, the dual in world coordinates.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "oca_solvers.cuh"

using namespace oca;

struct Stats {
    double dy = 0.0;
    long n = 0, bad = 0;
};

// one pair: a part with nr faces (box, or a regular polygon when poly > 0),
// an obstacle of no faces around a random centre, a random pose, proximal
// centre ybar and right-hand side bq
template <typename T, int D, int NR>
void one_pair(std::mt19937_64 &g, int poly, int FO, double spread, Stats &st) {
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::normal_distribution<double> G(0.0, 1.0);
    const int FR = NR;
    const T prox = T(1);
    int nr;
    std::vector<T> A(FR * D, T(0)), b(FR, T(1));
    if (poly > 0 && D == 2) {
        nr = poly;
        for (int k = 0; k < nr; ++k) {
            const double a = 2.0 * M_PI * k / nr;
            A[k * D] = T(std::cos(a));
            A[k * D + 1] = T(std::sin(a));
            b[k] = T(1);
        }
    } else {
        nr = 2 * D;
        for (int i = 0; i < D; ++i) {
            const double h = 0.3 + 2.0 * U(g);
            A[(2 * i) * D + i] = T(1);
            A[(2 * i + 1) * D + i] = T(-1);
            b[2 * i] = b[2 * i + 1] = T(h);
        }
    }
    T rho[D], R[D * D];
    for (int i = 0; i < D; ++i) rho[i] = T(spread * (U(g) - 0.5));
    if (D == 2) {
        const double th = 2.0 * M_PI * U(g);
        R[0] = T(std::cos(th));
        R[1] = T(-std::sin(th));
        R[2] = T(std::sin(th));
        R[3] = T(std::cos(th));
    } else {
        double M[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i][j] = G(g);
        for (int j = 0; j < 3; ++j) {  // Gram-Schmidt on the columns
            for (int k = 0; k < j; ++k) {
                double dd = 0.0;
                for (int i = 0; i < 3; ++i) dd += M[i][j] * M[i][k];
                for (int i = 0; i < 3; ++i) M[i][j] -= dd * M[i][k];
            }
            double nn = 0.0;
            for (int i = 0; i < 3; ++i) nn += M[i][j] * M[i][j];
            for (int i = 0; i < 3; ++i) M[i][j] /= std::sqrt(nn);
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) R[i * 3 + j] = T(M[i][j]);
    }
    const int no = std::max(D + 1, 3 + (int)(U(g) * (FO - 2)));
    std::vector<T> C(FO * D, T(0)), d(FO, T(1));
    double c0[3];
    for (int i = 0; i < D; ++i) c0[i] = 1.5 * spread * (U(g) - 0.5);
    for (int m = 0; m < no; ++m) {
        double nv[3] = {0.0, 0.0, 0.0}, nn = 0.0;
        if (D == 2) {
            const double a = 2.0 * M_PI * (m + 0.8 * U(g)) / no;  // spanning, sorted angles
            nv[0] = std::cos(a);
            nv[1] = std::sin(a);
            nn = 1.0;
        } else {
            for (int i = 0; i < 3; ++i) {
                nv[i] = G(g);
                nn += nv[i] * nv[i];
            }
            nn = std::sqrt(nn);
        }
        double cc = 0.0;
        for (int i = 0; i < D; ++i) {
            C[m * D + i] = T(nv[i] / nn);
            cc += double(C[m * D + i]) * c0[i];
        }
        d[m] = T(cc + 0.5 + 1.5 * U(g));
    }
    std::vector<T> yb(FR + FO + 1, T(0));
    for (int k = 0; k < nr; ++k) yb[k] = U(g) < 0.5 ? T(U(g)) : T(0);
    for (int m = 0; m < no; ++m) yb[FR + m] = U(g) < 0.4 ? T(0.5 * U(g)) : T(0);
    yb[FR + FO] = U(g) < 0.3 ? T(U(g)) : T(0);
    T bq[D + 1];
    bq[0] = T(1.0 + 0.4 * G(g));
    for (int i = 0; i < D; ++i) bq[1 + i] = T(0.4 * G(g));

    // unstaged body-frame solve from K^T ybar + bq
    Lane<T, D> L;
    for (int i = 0; i < D; ++i) L.rho[i] = rho[i];
    for (int i = 0; i < D * D; ++i) L.R[i] = R[i];
    L.A = A.data();
    L.b = b.data();
    L.nr = nr;
    L.C = C.data();
    L.d = d.data();
    L.no = no;
    T w[D + 1];
    for (int i = 0; i <= D; ++i) w[i] = bq[i];
    for (int k = 0; k < nr; ++k)
        for (int i = 0; i < D; ++i) w[1 + i] += yb[k] * A[k * D + i];
    for (int m = 0; m < no; ++m) {
        T gv[D + 1];
        gen_vec<T, D>(L, nr + m, gv);
        for (int i = 0; i <= D; ++i) w[i] += yb[FR + m] * gv[i];
    }
    w[0] += yb[FR + FO];
    SsnState<T, D> ref;
    const int s_ref = ssn_solve<T, D>(L, yb.data(), 1, FR, FO, prox, bq, w, ref);
    T u[D];
    for (int i = 0; i < D; ++i) {
        T acc = T(0);
        for (int k = 0; k < D; ++k) acc += R[i * D + k] * w[1 + k];
        u[i] = acc;
    }
    std::vector<T> y_ref(nr + no + 1);
    for (int gi = 0; gi < nr + no + 1; ++gi)
        y_ref[gi] = ssn_value<T, D>(L, yb.data(), 1, FR, FO, prox, w, u, ref.tau, gi);

    // staged world-frame solve, staged as the pair kernel stages it
    constexpr int NC = NrmStride<D>::N;
    SsnLane<T, D, NR> SL;
    SL.nr = nr;
    for (int k = 0; k < NR; ++k) {  // the breakpoint form; k >= nr is padding
        T a2 = T(0);
        for (int i = 0; i < D; ++i) a2 += A[k * D + i] * A[k * D + i];
        const T bk = k < nr ? b[k] : T(1);
        if (!(a2 > T(0))) a2 = T(1);
        for (int i = 0; i < D; ++i) {
            T acc = T(0);
            for (int l = 0; l < D; ++l) acc += R[i * D + l] * A[k * D + l];
            SL.ta[k][i] = acc / (prox * bk);
        }
        SL.bD[k] = k < nr ? bk / a2 : T(0);
        SL.w[k] = bk * SL.bD[k];
        SL.ty[k] = T(-3.0e38);
    }
    std::vector<T> nrm(FO * NC, T(0)), rec(4 * FO, T(0));
    T a0[D] = {}, w0[D] = {}, del0 = T(0);
    for (int k = 0; k < nr; ++k) {
        SL.ty[k] = yb[k] * m_rcp(SL.bD[k]);
        for (int i = 0; i < D; ++i) a0[i] += (prox * SL.w[k] * SL.ty[k]) * SL.ta[k][i];
    }
    for (int m = 0; m < no; ++m) {
        T cr = T(0), c2 = T(0);
        for (int i = 0; i < D; ++i) {
            const T c = C[m * D + i];
            nrm[m * NC + i] = c;
            cr += c * rho[i];
            c2 += c * c;
            w0[i] += yb[FR + m] * c;
        }
        del0 += yb[FR + m] * d[m];
        const T dp = d[m] - cr, pD = prox * (dp * dp + c2);
        rec_store<T>(rec.data() + 4 * m, dp, m_rcp(pD), yb[FR + m] * pD, yb[FR + m]);
    }
    SL.no = no;
    SL.rec = rec.data();
    SL.nrm = nrm.data();
    SL.ybg = yb[FR + FO];
    del0 += SL.ybg;
    T bqw[D + 1], ws[D + 1];
    bqw[0] = bq[0];
    for (int i = 0; i < D; ++i) {
        T acc = T(0);
        for (int k = 0; k < D; ++k) acc += R[i * D + k] * bq[1 + k];
        bqw[1 + i] = acc;
    }
    T wr = T(0);
    for (int i = 0; i < D; ++i) wr += w0[i] * rho[i];
    ws[0] = bqw[0] + del0 - wr;
    for (int i = 0; i < D; ++i) ws[1 + i] = bqw[1 + i] + a0[i] + w0[i];
    SsnKeep<T, NR> keep;
    const int s_new = ssn_solve_staged<T, D, NR>(SL, prox, T(1) / prox, bqw, ws, keep);
    std::vector<T> y_new(nr + no + 1);
    for (int k = 0; k < nr; ++k) y_new[k] = SL.bD[k] * keep.x[k];
    for (int m = 0; m < no; ++m) {
        T dp, iD, s, ybm, c[D];
        rec_load<T>(rec.data() + 4 * m, dp, iD, s, ybm);
        nrm_load<T, D>(nrm.data() + m * NC, c);
        T cw = T(0);
        for (int i = 0; i < D; ++i) cw += c[i] * ws[1 + i];
        y_new[nr + m] = std::fmax(T(0), (s - (ws[0] * dp + cw)) * iD);
    }
    y_new[nr + no] = std::fmax(T(0), SL.ybg - ws[0] / prox);

    double dy = 0.0, sc = 1.0;
    for (int i = 0; i < nr + no + 1; ++i) {
        dy = std::max(dy, std::fabs(double(y_new[i]) - double(y_ref[i])));
        sc = std::max(sc, std::fabs(double(y_ref[i])));
    }
    st.dy = std::max(st.dy, dy / sc);
    st.n += 1;
    if (s_new != OCA_PAIR_OK || s_ref != OCA_PAIR_OK) st.bad += 1;
}

template <typename T, int D, int NR>
void run(const char *name, int n, int poly, int FO, double spread, unsigned seed) {
    std::mt19937_64 g(seed);
    Stats st;
    for (int i = 0; i < n; ++i) one_pair<T, D, NR>(g, poly, FO, spread, st);
    std::printf("%s %ld %.3e %ld\n", name, st.n, st.dy, st.bad);
}

int main() {
    run<double, 2, 4>("f64_2d_box", 20000, 0, 16, 8.0, 11);
    run<float, 2, 4>("f32_2d_box", 20000, 0, 16, 8.0, 12);
    run<double, 3, 6>("f64_3d_box", 10000, 0, 20, 8.0, 13);
    run<float, 3, 6>("f32_3d_box", 10000, 0, 20, 8.0, 14);
    // a regular octagon part against obstacles of up to 24 faces, near and up
    // to 90 m away (large d', so a large rounding scale of psi): robot-face
    // sets with ties, where an Armijo slack that admits a real rise of psi
    // lets the iteration cycle between two sets
    run<double, 2, 8>("f64_2d_octagon", 20000, 8, 24, 8.0, 15);
    run<float, 2, 8>("f32_2d_octagon", 20000, 8, 24, 8.0, 16);
    run<float, 2, 8>("f32_2d_octagon_far", 40000, 8, 24, 120.0, 17);
    return 0;
}
