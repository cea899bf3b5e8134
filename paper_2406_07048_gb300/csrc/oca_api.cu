// Host side of the C-ABI declared in include/oca.h: argument checking, scene
// preparation (metadata, work tiles, workspace), kernel orchestration and the
// ADMM iteration driver (CUDA-graph chunks of iterations, per-scenario
// retirement on the device, host check between chunks).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "oca_common.cuh"
#include "oca_kernels.h"

using namespace oca;

struct oca_ctx {
    int device;
    int n_sm;
    int smem_optin;  // largest dynamic shared memory per block (opt-in), bytes
    // kernel timing (oca_profile_enable)
    bool prof = false;
    cudaEvent_t ev[4][8] = {};  // [pair start, pair stop, traj start, traj stop][iteration in chunk]
    double pair_ms = 0, traj_ms = 0;
    long long pair_launches = 0, traj_launches = 0;
};

struct oca_scene {
    oca_ctx *ctx = nullptr;
    int dim = 0, dtype = 0, S = 0, FO = 0, FR = 0, M_tot = 0, P_tot = 0;
    std::vector<ScenMeta> meta;
    std::vector<int64_t> pair_begin, state_begin, ctrl_begin;
    int64_t P = 0, n_states = 0, n_ctrls = 0;
    int Qtot = 0, maxQ = 0, n_tiles = 0, ny_max = 0, W = 1, maxN = 0;
    const void *obs_C = nullptr, *obs_d = nullptr, *part_A = nullptr, *part_b = nullptr, *part_off = nullptr;
    // device
    ScenMeta *d_meta = nullptr;
    Tile *d_tiles = nullptr;
    int *d_obs_nf = nullptr, *d_part_nf = nullptr, *d_part_link = nullptr;
    double *d_part_radius = nullptr;
    void *d_pose = nullptr, *d_stats = nullptr, *d_y2 = nullptr, *d_ric = nullptr;
    double *d_res = nullptr;
    long long *d_ric_off = nullptr;
    int *d_status = nullptr, *d_iter = nullptr, *d_active = nullptr, *d_err = nullptr;
    void *d_box = nullptr;      // z_s, w_s [n_states][NSmax]; z_u, w_u [n_ctrls][NUmax]
    int *d_mpc_i = nullptr;     // closed loop: per-step report (iters, status) [2][S]
    double *d_mpc_f = nullptr;  // per-step report (r_pri, r_dual, cost) [3][S] (scene dtype)
    unsigned char *d_mask = nullptr;  // [M_tot] sensed obstacles
    double *d_box_res = nullptr;  // [S][2]
    int *d_rev_iters = nullptr;   // fixed-point adjoint: reverse steps per scenario [S]
    int ns_max = 0, nu_max = 0;
    int *h_active = nullptr;
};

namespace {

#define OCA_CK(x)                                  \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return OCA_ERR_CUDA; \
    } while (0)

size_t dsize(int dtype) { return dtype == OCA_F64 ? sizeof(double) : sizeof(float); }

template <typename T>
Geom<T> make_geom(const oca_scene *sc) {
    Geom<T> g;
    g.obs_C = static_cast<const T *>(sc->obs_C);
    g.obs_d = static_cast<const T *>(sc->obs_d);
    g.obs_nf = sc->d_obs_nf;
    g.part_A = static_cast<const T *>(sc->part_A);
    g.part_b = static_cast<const T *>(sc->part_b);
    g.part_nf = sc->d_part_nf;
    g.part_link = sc->d_part_link;
    g.part_off = static_cast<const T *>(sc->part_off);
    g.FO = sc->FO;
    g.FR = sc->FR;
    return g;
}

template <typename T>
DevModel<T> make_model(const oca_model *m) {
    DevModel<T> d;
    d.kind = m->kind;
    d.dt = T(m->dt);
    for (int i = 0; i < 8; ++i) d.p[i] = T(m->param[i]);
    for (int i = 0; i < 12; ++i) d.Qs[i] = T(m->Qs[i]);
    for (int i = 0; i < 4; ++i) d.Qu[i] = T(m->Qu[i]);
    auto cl = [](double v) { return T(v < -1e30 ? -1e30 : (v > 1e30 ? 1e30 : v)); };
    for (int i = 0; i < 12; ++i) {
        d.s_lo[i] = cl(m->s_lo[i]);
        d.s_hi[i] = cl(m->s_hi[i]);
    }
    for (int i = 0; i < 4; ++i) {
        d.u_lo[i] = cl(m->u_lo[i]);
        d.u_hi[i] = cl(m->u_hi[i]);
    }
    return d;
}

int model_ns(int kind) { return kind == 0 ? 4 : kind == 1 ? 5 : 12; }

// the pair kernels' shared memory for W warps per tile (the largest form:
// ADMM mode with the Newton solver's staging) fits the device's per-block limit
bool warps_fit(const oca_scene *sc, int W) {
    return W <= pair_max_warps(sc->dim, dsize(sc->dtype)) &&
           pair_smem_bytes(sc->dim, dsize(sc->dtype), W, 1, 1, sc->FR, sc->FO) <= (size_t)sc->ctx->smem_optin;
}

oca_status check_model(const oca_scene *sc, const oca_model *m) {
    if (!m || m->kind < 0 || m->kind > 2) return OCA_ERR_INVALID_ARGUMENT;
    if ((m->kind == 2) != (sc->dim == 3)) return OCA_ERR_INVALID_ARGUMENT;
    if (!(m->dt > 0.0) || !std::isfinite(m->dt)) return OCA_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < 12; ++i)
        if (std::isnan(m->s_lo[i]) || std::isnan(m->s_hi[i]) || m->s_lo[i] > m->s_hi[i]) return OCA_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < 4; ++i)
        if (std::isnan(m->u_lo[i]) || std::isnan(m->u_hi[i]) || m->u_lo[i] > m->u_hi[i]) return OCA_ERR_INVALID_ARGUMENT;
    return OCA_OK;
}

// ---- scene validation: part offsets positive, geometry finite; radius of
// each part (largest vertex norm, by enumerating dim-subsets of faces) for the
// certificate margin.
template <typename T>
__global__ void k_validate(const T *obs_C, const T *obs_d, const int *obs_nf, int M_tot, const T *part_A,
                           const T *part_b, const int *part_nf, int P_tot, const T *part_off, int FO, int FR,
                           int dim, double *radius, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M_tot) {
        const int nf = obs_nf[i];
        for (int k = 0; k < nf * dim; ++k)
            if (!isfinite(double(obs_C[(long long)i * FO * dim + k]))) atomicOr(err, 1);
        for (int k = 0; k < nf; ++k)
            if (!isfinite(double(obs_d[(long long)i * FO + k]))) atomicOr(err, 1);
    }
    if (i < P_tot) {
        const int nr = part_nf[i];
        const T *A = part_A + (long long)i * FR * dim;
        const T *b = part_b + (long long)i * FR;
        for (int k = 0; k < nr; ++k) {
            if (!(double(b[k]) > 0.0) || !isfinite(double(b[k]))) atomicOr(err, 2);
            for (int l = 0; l < dim; ++l)
                if (!isfinite(double(A[k * dim + l]))) atomicOr(err, 2);
        }
        for (int l = 0; l < dim; ++l)
            if (!isfinite(double(part_off[(long long)i * dim + l]))) atomicOr(err, 2);
        double rmax = 0.0;
        int nv = 0;
        for (int a = 0; a < nr; ++a)
            for (int b2 = a + 1; b2 < nr; ++b2)
                for (int c = (dim == 3 ? b2 + 1 : 0); c < (dim == 3 ? nr : 1); ++c) {
                    double x[3];
                    if (dim == 2) {
                        const double a00 = A[a * 2], a01 = A[a * 2 + 1], a10 = A[b2 * 2], a11 = A[b2 * 2 + 1];
                        const double det = a00 * a11 - a01 * a10;
                        if (fabs(det) < 1e-12) continue;
                        x[0] = (double(b[a]) * a11 - a01 * double(b[b2])) / det;
                        x[1] = (a00 * double(b[b2]) - double(b[a]) * a10) / det;
                    } else {
                        double M[3][3], r[3];
                        const int id[3] = {a, b2, c};
                        for (int u = 0; u < 3; ++u) {
                            for (int v = 0; v < 3; ++v) M[u][v] = A[id[u] * 3 + v];
                            r[u] = b[id[u]];
                        }
                        const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                                           M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                                           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
                        if (fabs(det) < 1e-12) continue;
                        for (int col = 0; col < 3; ++col) {
                            double Mc[3][3];
                            for (int u = 0; u < 3; ++u)
                                for (int v = 0; v < 3; ++v) Mc[u][v] = (v == col) ? r[u] : M[u][v];
                            x[col] = (Mc[0][0] * (Mc[1][1] * Mc[2][2] - Mc[1][2] * Mc[2][1]) -
                                      Mc[0][1] * (Mc[1][0] * Mc[2][2] - Mc[1][2] * Mc[2][0]) +
                                      Mc[0][2] * (Mc[1][0] * Mc[2][1] - Mc[1][1] * Mc[2][0])) / det;
                        }
                    }
                    bool feas = true;
                    for (int k = 0; k < nr && feas; ++k) {
                        double sacc = 0.0;
                        for (int l = 0; l < dim; ++l) sacc += double(A[k * dim + l]) * x[l];
                        if (sacc > double(b[k]) + 1e-9 * (1.0 + fabs(double(b[k])))) feas = false;
                    }
                    if (!feas) continue;
                    double n2 = 0.0;
                    for (int l = 0; l < dim; ++l) n2 += x[l] * x[l];
                    rmax = fmax(rmax, sqrt(n2));
                    ++nv;
                }
        if (nv < dim + 1) atomicOr(err, 4);  // unbounded or degenerate part
        radius[i] = rmax;
    }
}

__global__ void k_reset(int *status, int S, int *iter, int *active) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S) status[i] = kActive;
    if (i == 0) {
        *iter = 0;
        *active = S;
    }
}

__global__ void k_advance(int *iter) { *iter += 1; }

// box block initial state: z = clip(s or u), w = 0 (bounds passed by value)
template <typename T>
struct Bounds12 {
    T lo[12], hi[12];
};

template <typename T>
__global__ void k_box_init(const T *x, long long n, int nc, Bounds12<T> b, T *z, T *w) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nc) return;
    const int c = (int)(i % nc);
    z[i] = fmin(fmax(x[i], b.lo[c]), b.hi[c]);
    w[i] = T(0);
}

// final y of a scenario retired at iteration j lives in buffer j % 2
// y of the scenarios whose last iteration left it in the second buffer back
// into the caller's y: only a pair's own components (lambda_k, k < n_faces
// of the part; mu_m, m < n_faces of the obstacle; gamma), padding untouched
template <typename T>
__global__ void k_gather(const ScenMeta *meta, const int *iters, const int *part_nf, const int *obs_nf, int FR, int FO,
                         const T *y2, T *y, long long P, int ny) {
    const int s = blockIdx.y;
    if (!(iters[s] & 1)) return;
    const ScenMeta sm = meta[s];
    const long long np = (long long)sm.M * sm.NP * sm.N;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < np * ny; k += (long long)gridDim.x * blockDim.x) {
        const long long c = k / np, l = k % np, p = sm.pair0 + l;
        const int j = (int)(l / ((long long)sm.NP * sm.N)), part = (int)((l / sm.N) % sm.NP);
        const bool own = c < FR ? c < part_nf[sm.part0 + part]
                                : (c < FR + FO ? c - FR < obs_nf[sm.obs0 + j] : true);
        if (own) y[c * P + p] = y2[c * P + p];
    }
}

template <typename T>
oca_status scale_impl(oca_scene *sc, const oca_model *m, const void *states, void *alpha, void *lambda, void *mu,
                      double *margin, int32_t *verdict, int32_t *status, cudaStream_t st) {
    PoseArgs<T> pa;
    pa.meta = sc->d_meta;
    pa.n_scen = sc->S;
    pa.g = make_geom<T>(sc);
    pa.model = make_model<T>(m);
    pa.states = static_cast<const T *>(states);
    pa.pose = static_cast<T *>(sc->d_pose);
    pa.Qtot = sc->Qtot;
    pa.scen_status = nullptr;
    OCA_CK(launch_pose<T>(pa, sc->maxQ, st));
    ScaleArgs<T> a;
    a.meta = sc->d_meta;
    a.tiles = sc->d_tiles;
    a.g = make_geom<T>(sc);
    a.pose = static_cast<const T *>(sc->d_pose);
    a.Qtot = sc->Qtot;
    a.P = sc->P;
    a.part_radius = sc->d_part_radius;
    a.alpha = static_cast<T *>(alpha);
    a.lambda = static_cast<T *>(lambda);
    a.mu = static_cast<T *>(mu);
    a.margin = margin;
    a.verdict = verdict;
    a.status = status;
    OCA_CK(launch_scale<T>(a, sc->dim, sc->n_tiles, sc->W, st));
    return OCA_OK;
}

template <typename T>
oca_status cert_impl(oca_scene *sc, const oca_model *m, const void *states, const void *lambda, const void *mu,
                     double *margin, cudaStream_t st) {
    CertArgs<T> a;
    a.meta = sc->d_meta;
    a.tiles = sc->d_tiles;
    a.g = make_geom<T>(sc);
    a.model = make_model<double>(m);
    a.states = static_cast<const T *>(states);
    a.P = sc->P;
    a.part_radius = sc->d_part_radius;
    a.lambda = static_cast<const T *>(lambda);
    a.mu = static_cast<const T *>(mu);
    a.margin = margin;
    OCA_CK(launch_cert<T>(a, sc->n_tiles, sc->W, st));
    return OCA_OK;
}

template <typename T>
PairArgs<T> pair_args(oca_scene *sc) {
    PairArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.meta = sc->d_meta;
    a.tiles = sc->d_tiles;
    a.g = make_geom<T>(sc);
    a.pose = static_cast<const T *>(sc->d_pose);
    a.Qtot = sc->Qtot;
    a.P = sc->P;
    a.res = sc->d_res;
    a.n_tiles = sc->n_tiles;
    a.stats = static_cast<T *>(sc->d_stats);
    return a;
}

template <typename T>
oca_status pairqp_impl(oca_scene *sc, const oca_model *m, const void *states, const void *zeta, const void *xi,
                       double prox, const void *y_in, void *y_out, void *v_out, void *obj_out, int32_t *status_out,
                       cudaStream_t st) {
    PoseArgs<T> pa;
    pa.meta = sc->d_meta;
    pa.n_scen = sc->S;
    pa.g = make_geom<T>(sc);
    pa.model = make_model<T>(m);
    pa.states = static_cast<const T *>(states);
    pa.pose = static_cast<T *>(sc->d_pose);
    pa.Qtot = sc->Qtot;
    pa.scen_status = nullptr;
    OCA_CK(launch_pose<T>(pa, sc->maxQ, st));
    PairArgs<T> a = pair_args<T>(sc);
    a.zeta = const_cast<T *>(static_cast<const T *>(zeta));
    a.xi = const_cast<T *>(static_cast<const T *>(xi));
    a.y_in = static_cast<const T *>(y_in);
    a.y_out = static_cast<T *>(y_out);
    a.v_out = static_cast<T *>(v_out);
    a.obj_out = static_cast<T *>(obj_out);
    a.status_out = status_out;
    a.prox = T(prox);
    OCA_CK(launch_pair<T>(a, sc->dim, 0, prox > 0.0 ? 1 : 0, sc->n_tiles, sc->W, st));
    return OCA_OK;
}


// ---- tape of a solve for the adjoint: iterates, then the backward pass's
// work area.  Offsets in elements of the scene dtype (regions 256-byte
// aligned); the two double accumulators come last.
struct TapeLayout {
    long long y, zx, st, s, u, box;                   // iterate regions
    long long y_slot, zx_slot, st_slot, s_slot, u_slot, box_slot;
    long long yb, zb, sb, ub, bb, stb, pb, sf;        // adjoint work area
    long long work_end;                               // end of the T regions
    size_t gd_byte, gs0_byte, bytes;
};

// fp (OCA_ADMM_FIXED_POINT): one slot of every iterate region (the final
// iterate), whatever K is
TapeLayout tape_layout(const oca_scene *sc, int kind, int K, bool fp = false) {
    const int NS = kind == 0 ? 4 : kind == 1 ? 5 : 12, NU = kind == 2 ? 4 : 2;
    const int D = sc->dim, NSTAT = D * (D + 1) / 2 + D + D * D, PK = D + D * D;
    const long long es = (long long)dsize(sc->dtype);
    const long long al = 256 / es;
    auto up = [&](long long x) { return (x + al - 1) / al * al; };
    TapeLayout L;
    L.y_slot = up((long long)sc->ny_max * sc->P);
    L.zx_slot = up((long long)(1 + D) * sc->P);
    L.st_slot = up((long long)NSTAT * sc->Qtot);
    L.s_slot = up(sc->n_states * NS);
    L.u_slot = up(sc->n_ctrls * NU);
    L.box_slot = up(2 * sc->n_states * NS + 2 * sc->n_ctrls * NU);
    const long long n1 = fp ? 1 : (long long)K + 1, n0 = fp ? 1 : (long long)K;  // slots
    long long o = 0;
    L.y = o;   o += n1 * L.y_slot;
    L.zx = o;  o += n0 * L.zx_slot;
    L.st = o;  o += n0 * L.st_slot;
    L.s = o;   o += n1 * L.s_slot;
    L.u = o;   o += n1 * L.u_slot;
    L.box = o; o += n1 * L.box_slot;
    L.yb = o;  o += 2 * L.y_slot;
    L.zb = o;  o += L.zx_slot;
    L.sb = o;  o += L.s_slot;
    L.ub = o;  o += L.u_slot;
    L.bb = o;  o += L.box_slot;
    L.stb = o; o += L.st_slot;
    L.pb = o;  o += up((long long)PK * sc->Qtot);
    L.sf = o;  o += L.s_slot;
    L.work_end = o;
    size_t b = (size_t)o * (size_t)es;
    b = (b + 255) / 256 * 256;
    L.gd_byte = b;
    b += sizeof(double) * (size_t)sc->M_tot * sc->FO;
    b = (b + 255) / 256 * 256;
    L.gs0_byte = b;
    b += sizeof(double) * (size_t)sc->S * NS;
    L.bytes = (b + 255) / 256 * 256;
    return L;
}

template <typename T>
__global__ void k_cast_d2t(const double *x, long long n, T *y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = T(x[i]);
}


template <typename T>
oca_status lemke_impl(oca_scene *sc, const oca_model *m, const void *states, const void *zeta, const void *xi,
                      double prox, const void *y_in, void *y_out, void *v_out, void *obj_out, int32_t *status_out,
                      cudaStream_t st) {
    PoseArgs<T> pa;
    pa.meta = sc->d_meta;
    pa.n_scen = sc->S;
    pa.g = make_geom<T>(sc);
    pa.model = make_model<T>(m);
    pa.states = static_cast<const T *>(states);
    pa.pose = static_cast<T *>(sc->d_pose);
    pa.Qtot = sc->Qtot;
    pa.scen_status = nullptr;
    OCA_CK(launch_pose<T>(pa, sc->maxQ, st));
    LemkeArgs<T> a;
    a.meta = sc->d_meta;
    a.g = make_geom<T>(sc);
    a.pose = static_cast<const T *>(sc->d_pose);
    a.Qtot = sc->Qtot;
    a.P = sc->P;
    a.n_scen = sc->S;
    a.zeta = static_cast<const T *>(zeta);
    a.xi = static_cast<const T *>(xi);
    a.y_in = static_cast<const T *>(y_in);
    a.y_out = static_cast<T *>(y_out);
    a.v_out = static_cast<T *>(v_out);
    a.obj_out = static_cast<T *>(obj_out);
    a.status_out = status_out;
    a.prox = T(prox);
    OCA_CK(launch_lemke<T>(a, sc->dim, st));
    return OCA_OK;
}

template <typename T>
oca_status admm_impl(oca_scene *sc, const oca_model *m, const oca_admm_params *pr, const void *s_ref, void *s,
                     void *u, void *y, void *zeta, void *xi, const oca_admm_report *rep, cudaStream_t st,
                     void *tape = nullptr, const unsigned char *obs_mask = nullptr,
                     cudaGraphExec_t *graph_cache = nullptr, bool host_stop = true) {
    k_reset<<<(sc->S + 255) / 256, 256, 0, st>>>(sc->d_status, sc->S, sc->d_iter, sc->d_active);
    OCA_CK(cudaGetLastError());
    const int NS = model_ns(m->kind), NU = m->kind == 2 ? 4 : 2;
    T *box = static_cast<T *>(sc->d_box);
    T *zs = box, *ws = zs + (size_t)sc->n_states * sc->ns_max;
    T *zu = ws + (size_t)sc->n_states * sc->ns_max, *wu = zu + (size_t)sc->n_ctrls * sc->nu_max;
    {
        const DevModel<T> dm = make_model<T>(m);
        Bounds12<T> bs, bu;
        for (int i = 0; i < 12; ++i) {
            bs.lo[i] = dm.s_lo[i];
            bs.hi[i] = dm.s_hi[i];
            bu.lo[i] = i < 4 ? dm.u_lo[i] : T(0);
            bu.hi[i] = i < 4 ? dm.u_hi[i] : T(0);
        }
        const long long n1 = sc->n_states * NS, n2 = sc->n_ctrls * NU;
        k_box_init<T><<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(static_cast<const T *>(s), sc->n_states, NS, bs, zs, ws);
        k_box_init<T><<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(static_cast<const T *>(u), sc->n_ctrls, NU, bu, zu, wu);
        OCA_CK(cudaGetLastError());
        OCA_CK(cudaMemsetAsync(sc->d_box_res, 0, sizeof(double) * 2 * sc->S, st));
    }
    PoseArgs<T> pa;
    pa.meta = sc->d_meta;
    pa.n_scen = sc->S;
    pa.g = make_geom<T>(sc);
    pa.model = make_model<T>(m);
    pa.states = static_cast<const T *>(s);
    pa.pose = static_cast<T *>(sc->d_pose);
    pa.Qtot = sc->Qtot;
    pa.scen_status = nullptr;
    OCA_CK(launch_pose<T>(pa, sc->maxQ, st));

    // tape (oca_admm_solve_taped): iterate 0 now, iterate j+1 after launch j;
    // a fixed-point tape (OCA_ADMM_FIXED_POINT) takes the final iterate only,
    // after the solve, which then runs as an untaped one
    TapeLayout TL{};
    const bool fp_tape = tape && (pr->flags & OCA_ADMM_FIXED_POINT);
    T *tp = fp_tape ? nullptr : static_cast<T *>(tape);
    const size_t es = sizeof(T);
    const size_t box_s = (size_t)sc->n_states * NS, box_u = (size_t)sc->n_ctrls * NU;
    auto tape_box = [&](int slot) -> cudaError_t {
        T *dst = tp + TL.box + (long long)slot * TL.box_slot;
        cudaError_t e = cudaMemcpyAsync(dst, zs, es * box_s, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst + box_s, ws, es * box_s, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst + 2 * box_s, zu, es * box_u, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst + 2 * box_s + box_u, wu, es * box_u, cudaMemcpyDeviceToDevice, st);
        return e;
    };
    if (tp) {
        TL = tape_layout(sc, m->kind, pr->max_iter);
        OCA_CK(cudaMemcpyAsync(tp + TL.y, y, es * sc->ny_max * (size_t)sc->P, cudaMemcpyDeviceToDevice, st));
        OCA_CK(cudaMemcpyAsync(tp + TL.s, s, es * box_s, cudaMemcpyDeviceToDevice, st));
        OCA_CK(cudaMemcpyAsync(tp + TL.u, u, es * box_u, cudaMemcpyDeviceToDevice, st));
        OCA_CK(tape_box(0));
    }

    PairArgs<T> a = pair_args<T>(sc);
    a.zeta = static_cast<T *>(zeta);
    a.xi = static_cast<T *>(xi);
    a.y_in = static_cast<const T *>(y);
    a.y_out = static_cast<T *>(sc->d_y2);
    a.scen_status = sc->d_status;
    a.iter = sc->d_iter;
    a.max_iter = pr->max_iter;
    a.prox = T(pr->prox);
    a.obs_mask = obs_mask;
    const int solver = pr->prox > 0.0 ? 1 : 0;

    RicArgs<T> r;
    r.meta = sc->d_meta;
    r.n_scen = sc->S;
    r.g = make_geom<T>(sc);
    r.model = make_model<T>(m);
    r.sigma = T(pr->sigma);
    r.eps_pri = T(pr->eps_pri);
    r.eps_dual = T(pr->eps_dual);
    r.rho_box = T(pr->rho_box);
    r.damp = T(pr->damp);
    r.box_zs = zs;
    r.box_ws = ws;
    r.box_zu = zu;
    r.box_wu = wu;
    r.box_res = sc->d_box_res;
    r.max_iter = pr->max_iter;
    r.iter = sc->d_iter;
    r.s_ref = static_cast<const T *>(s_ref);
    r.s = static_cast<T *>(s);
    r.u = static_cast<T *>(u);
    r.pose = static_cast<T *>(sc->d_pose);
    r.stats = static_cast<const T *>(sc->d_stats);
    r.Qtot = sc->Qtot;
    r.res = sc->d_res;
    r.n_tiles = sc->n_tiles;
    r.scen_status = sc->d_status;
    r.iters_out = rep->iters;
    r.status_out = rep->status;
    r.r_pri_out = static_cast<T *>(rep->r_pri);
    r.r_dual_out = static_cast<T *>(rep->r_dual);
    r.cost_out = static_cast<T *>(rep->cost);
    r.active_count = sc->d_active;
    r.scratch = sc->d_ric;
    r.scratch0 = sc->d_ric_off;
    const bool f32 = (pr->flags & OCA_ADMM_RICCATI_F32) != 0 && sizeof(T) == sizeof(float);

    oca_ctx *cx = sc->ctx;
    const bool prof = cx->prof;
    bool capturing = false;
    auto rec = [&](cudaEvent_t e) -> cudaError_t {
        return capturing ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
    };
    auto one_iter = [&](int k, long long j) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (prof && (e = rec(cx->ev[0][k])) != cudaSuccess) return e;
        e = launch_pair<T>(a, sc->dim, 1, solver, sc->n_tiles, sc->W, st);
        if (e != cudaSuccess) return e;
        if (prof && (e = rec(cx->ev[1][k])) != cudaSuccess) return e;
        const bool rec_tape = tp && j < pr->max_iter;
        if (rec_tape) {
            // y^{j+1} sits in the buffer launch j wrote; zeta^j, xi^j after its head
            const T *ynew = (j & 1) ? static_cast<const T *>(y) : static_cast<const T *>(sc->d_y2);
            e = cudaMemcpyAsync(tp + TL.y + (j + 1) * TL.y_slot, ynew, es * sc->ny_max * (size_t)sc->P,
                                cudaMemcpyDeviceToDevice, st);
            T *zx = tp + TL.zx + j * TL.zx_slot;
            if (e == cudaSuccess) e = cudaMemcpyAsync(zx, zeta, es * (size_t)sc->P, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(zx + sc->P, xi, es * sc->dim * (size_t)sc->P, cudaMemcpyDeviceToDevice, st);
            const int nstat = sc->dim * (sc->dim + 1) / 2 + sc->dim + sc->dim * sc->dim;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(tp + TL.st + j * TL.st_slot, sc->d_stats, es * nstat * (size_t)sc->Qtot,
                                    cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        }
        if (prof && (e = rec(cx->ev[2][k])) != cudaSuccess) return e;
        e = launch_riccati<T>(r, f32, st);
        if (e != cudaSuccess) return e;
        if (prof && (e = rec(cx->ev[3][k])) != cudaSuccess) return e;
        if (rec_tape) {
            e = cudaMemcpyAsync(tp + TL.s + (j + 1) * TL.s_slot, s, es * box_s, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(tp + TL.u + (j + 1) * TL.u_slot, u, es * box_u, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = tape_box((int)(j + 1));
            if (e != cudaSuccess) return e;
        }
        k_advance<<<1, 1, 0, st>>>(sc->d_iter);
        return cudaGetLastError();
    };
    const int G = 8;  // iterations per chunk between host checks
    const long long n_launch = (long long)pr->max_iter + 1;  // j = 0..max_iter
    // graph_cache: a caller that solves repeatedly with the same arguments
    // (the closed loop) keeps the instantiated graph between calls
    cudaGraphExec_t exec = graph_cache ? *graph_cache : nullptr;
    if (!exec && st != nullptr && n_launch > G && !tp) {
        cudaGraph_t graph = nullptr;
        OCA_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        cudaError_t ce = cudaSuccess;
        for (int k = 0; k < G && ce == cudaSuccess; ++k) ce = one_iter(k, k);
        capturing = false;
        cudaError_t ee = cudaStreamEndCapture(st, &graph);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return OCA_ERR_CUDA;
        }
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return OCA_ERR_CUDA;
        if (graph_cache) *graph_cache = exec;
    }
    oca_status out = OCA_OK;
    *sc->h_active = sc->S;
    // host_stop: read the active count after every chunk and stop when no
    // scenario is left; without it (the closed loop, where some scenario
    // nearly always runs to the cap) every chunk is enqueued back to back and
    // chunks after the last retirement exit at once on the device.  Profiling
    // reads its per-chunk events, so it keeps the per-chunk wait.
    const bool wait_each = host_stop || prof;
    for (long long done = 0; done < n_launch; done += G) {
        if (exec) {
            if (cudaGraphLaunch(exec, st) != cudaSuccess) { out = OCA_ERR_CUDA; break; }
        } else {
            for (int k = 0; k < G && done + k < n_launch; ++k)
                if (one_iter(k, done + k) != cudaSuccess) { out = OCA_ERR_CUDA; break; }
            if (out != OCA_OK) break;
        }
        if (!wait_each) continue;
        if (cudaMemcpyAsync(sc->h_active, sc->d_active, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            out = OCA_ERR_CUDA;
            break;
        }
        if (prof) {
            const long long nk = std::min<long long>(G, n_launch - done);
            for (long long k = 0; k < nk; ++k) {
                float m1 = 0.f, m2 = 0.f;
                if (cudaEventElapsedTime(&m1, cx->ev[0][k], cx->ev[1][k]) != cudaSuccess ||
                    cudaEventElapsedTime(&m2, cx->ev[2][k], cx->ev[3][k]) != cudaSuccess) {
                    out = OCA_ERR_CUDA;
                    break;
                }
                cx->pair_ms += m1;
                cx->traj_ms += m2;
                cx->pair_launches += 1;
                cx->traj_launches += 1;
            }
            if (out != OCA_OK) break;
        }
        if (*sc->h_active <= 0) break;
    }
    if (exec && !graph_cache) cudaGraphExecDestroy(exec);
    if (out != OCA_OK) return out;
    dim3 gg(64, sc->S);
    k_gather<T><<<gg, 256, 0, st>>>(sc->d_meta, rep->iters, sc->d_part_nf, sc->d_obs_nf, sc->FR, sc->FO,
                                    static_cast<const T *>(sc->d_y2), static_cast<T *>(y), sc->P, sc->ny_max);
    OCA_CK(cudaGetLastError());
    if (fp_tape) {
        // the returned iterate of every scenario: y, zeta, xi, s, u as returned;
        // the statistics and the box block as its last iteration left them
        // (retired scenarios' entries are not touched after they retire)
        const TapeLayout FL = tape_layout(sc, m->kind, 0, true);
        T *ft = static_cast<T *>(tape);
        const int nstat = sc->dim * (sc->dim + 1) / 2 + sc->dim + sc->dim * sc->dim;
        OCA_CK(cudaMemcpyAsync(ft + FL.y, y, es * sc->ny_max * (size_t)sc->P, cudaMemcpyDeviceToDevice, st));
        OCA_CK(cudaMemcpyAsync(ft + FL.zx, zeta, es * (size_t)sc->P, cudaMemcpyDeviceToDevice, st));
        OCA_CK(cudaMemcpyAsync(ft + FL.zx + sc->P, xi, es * sc->dim * (size_t)sc->P, cudaMemcpyDeviceToDevice, st));
        OCA_CK(cudaMemcpyAsync(ft + FL.st, sc->d_stats, es * nstat * (size_t)sc->Qtot, cudaMemcpyDeviceToDevice, st));
        OCA_CK(cudaMemcpyAsync(ft + FL.s, s, es * box_s, cudaMemcpyDeviceToDevice, st));
        OCA_CK(cudaMemcpyAsync(ft + FL.u, u, es * box_u, cudaMemcpyDeviceToDevice, st));
        T *dst = ft + FL.box;
        OCA_CK(cudaMemcpyAsync(dst, zs, es * box_s, cudaMemcpyDeviceToDevice, st));
        OCA_CK(cudaMemcpyAsync(dst + box_s, ws, es * box_s, cudaMemcpyDeviceToDevice, st));
        OCA_CK(cudaMemcpyAsync(dst + 2 * box_s, zu, es * box_u, cudaMemcpyDeviceToDevice, st));
        OCA_CK(cudaMemcpyAsync(dst + 2 * box_s + box_u, wu, es * box_u, cudaMemcpyDeviceToDevice, st));
    }
    return OCA_OK;
}


__global__ void k_rev_iters(const int32_t *iters, int K, int S, int *out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) out[s] = iters[s] > 0 ? K : 0;
}

template <typename T>
oca_status backward_impl(oca_scene *sc, const oca_model *m, const oca_admm_params *pr, const void *s_ref, void *tape,
                         const int32_t *iters, const void *grad_cost, const void *grad_alpha, void *grad_d,
                         void *grad_ctr, void *grad_s0, cudaStream_t st) {
    const int K = pr->max_iter;
    const int NS = model_ns(m->kind), NU = m->kind == 2 ? 4 : 2;
    // fixed point: K reverse steps of the iteration map, all at the one taped
    // iterate (zero slot strides), for every scenario that ran an iteration
    const bool fp = (pr->flags & OCA_ADMM_FIXED_POINT) != 0;
    const TapeLayout TL = tape_layout(sc, m->kind, K, fp);
    if (fp) {
        k_rev_iters<<<(sc->S + 255) / 256, 256, 0, st>>>(iters, K, sc->S, sc->d_rev_iters);
        OCA_CK(cudaGetLastError());
        iters = sc->d_rev_iters;
    }
    T *tp = static_cast<T *>(tape);
    unsigned char *tb = static_cast<unsigned char *>(tape);
    // zero the work area and the accumulators
    OCA_CK(cudaMemsetAsync(tp + TL.yb, 0, TL.bytes - sizeof(T) * (size_t)TL.yb, st));
    double *gd = reinterpret_cast<double *>(tb + TL.gd_byte);
    double *gs0 = reinterpret_cast<double *>(tb + TL.gs0_byte);

    TapeView<T> tv;
    tv.y = tp + TL.y;
    tv.zx = tp + TL.zx;
    tv.stats = tp + TL.st;
    tv.s = tp + TL.s;
    tv.u = tp + TL.u;
    tv.box = tp + TL.box;
    tv.y_slot = fp ? 0 : TL.y_slot;
    tv.zx_slot = fp ? 0 : TL.zx_slot;
    tv.stats_slot = fp ? 0 : TL.st_slot;
    tv.s_slot = fp ? 0 : TL.s_slot;
    tv.u_slot = fp ? 0 : TL.u_slot;
    tv.box_slot = fp ? 0 : TL.box_slot;
    tv.n_states = sc->n_states;
    tv.n_ctrls = sc->n_ctrls;

    T *bb = tp + TL.bb;
    const long long box_s = sc->n_states * NS, box_u = sc->n_ctrls * NU;
    AdjTrajArgs<T> ta;
    std::memset(&ta, 0, sizeof(ta));
    ta.meta = sc->d_meta;
    ta.g = make_geom<T>(sc);
    ta.model = make_model<T>(m);
    ta.sigma = T(pr->sigma);
    ta.rho_box = T(pr->rho_box);
    ta.damp = T(pr->damp);
    ta.s_ref = static_cast<const T *>(s_ref);
    ta.Qtot = sc->Qtot;
    ta.iters = iters;
    ta.tape = tv;
    ta.grad_cost = static_cast<const T *>(grad_cost);
    ta.sb = tp + TL.sb;
    ta.ub = tp + TL.ub;
    ta.zsb = bb;
    ta.wsb = bb + box_s;
    ta.zub = bb + 2 * box_s;
    ta.wub = bb + 2 * box_s + box_u;
    ta.statsb = tp + TL.stb;
    ta.poseb = tp + TL.pb;
    ta.gs0 = gs0;
    ta.scratch = sc->d_ric;
    ta.scratch0 = sc->d_ric_off;
    OCA_CK(launch_adj_seed<T>(ta, sc->S, st));

    PoseArgs<T> pa;
    pa.meta = sc->d_meta;
    pa.n_scen = sc->S;
    pa.g = make_geom<T>(sc);
    pa.model = make_model<T>(m);
    pa.pose = static_cast<T *>(sc->d_pose);
    pa.Qtot = sc->Qtot;
    pa.scen_status = nullptr;
    const int W = std::min(sc->W, 8);
    if (grad_alpha) {
        // alpha* at the returned states seeds the pose adjoints and the offsets
        AdjAlphaArgs<T> aa;
        aa.meta = sc->d_meta;
        aa.tiles = sc->d_tiles;
        aa.g = make_geom<T>(sc);
        aa.pose = static_cast<const T *>(sc->d_pose);
        aa.Qtot = sc->Qtot;
        aa.P = sc->P;
        aa.grad_alpha = static_cast<const T *>(grad_alpha);
        aa.poseb = tp + TL.pb;
        aa.gd = gd;
        OCA_CK(launch_adj_alpha<T>(aa, sc->dim, sc->n_tiles, W, iters, tp + TL.s, tv.s_slot, NS, sc->S, tp + TL.sf, pa,
                                   sc->maxQ, st));
    }

    AdjPairArgs<T> ap;
    std::memset(&ap, 0, sizeof(ap));
    ap.meta = sc->d_meta;
    ap.tiles = sc->d_tiles;
    ap.g = make_geom<T>(sc);
    ap.pose = static_cast<const T *>(sc->d_pose);
    ap.Qtot = sc->Qtot;
    ap.P = sc->P;
    ap.prox = T(pr->prox);
    ap.iters = iters;
    ap.zb = tp + TL.zb;
    ap.xb = tp + TL.zb + sc->P;
    ap.statsb = tp + TL.stb;
    ap.poseb = tp + TL.pb;
    ap.gd = gd;
    for (int k = K - 1; k >= 0; --k) {
        ta.k = k;
        OCA_CK(launch_adj_traj<T>(ta, sc->S, st));
        pa.states = tp + TL.s + (long long)k * tv.s_slot;
        OCA_CK(launch_pose<T>(pa, sc->maxQ, st));
        ap.k = k;
        ap.y_k = tp + TL.y + (long long)k * tv.y_slot;
        ap.y_k1 = tp + TL.y + (long long)(k + 1) * tv.y_slot;
        ap.zx_k = tp + TL.zx + (long long)k * tv.zx_slot;
        ap.ybar_in = tp + TL.yb + (long long)((k + 1) & 1) * TL.y_slot;
        ap.ybar_out = tp + TL.yb + (long long)(k & 1) * TL.y_slot;
        OCA_CK(launch_adj_pair<T>(ap, sc->dim, sc->n_tiles, W, st));
    }
    OCA_CK(launch_adj_finish<T>(gd, static_cast<const T *>(sc->obs_C), sc->d_obs_nf, sc->M_tot, sc->FO, sc->dim,
                                static_cast<T *>(grad_d), static_cast<T *>(grad_ctr), st));
    if (grad_s0) {
        const long long n = (long long)sc->S * NS;
        k_cast_d2t<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(gs0, n, static_cast<T *>(grad_s0));
        OCA_CK(cudaGetLastError());
    }
    return OCA_OK;
}


template <typename T>
oca_status mpc_impl(oca_scene *sc, const oca_model *m, const oca_admm_params *pr, const oca_mpc_params *mp,
                    const void *ref, int T_ref, const void *obs_center, void *x, void *s_ref, void *s, void *u,
                    void *y, void *zeta, void *xi, void *x_hist, void *u_hist, int32_t *iters_hist,
                    int32_t *collided, cudaStream_t st) {
    MpcArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.meta = sc->d_meta;
    a.g = make_geom<T>(sc);
    a.model = make_model<T>(m);
    a.ref = static_cast<const T *>(ref);
    a.T_ref = T_ref;
    a.obs_center = static_cast<const T *>(obs_center);
    for (int i = 0; i < 3; ++i) a.win[i] = T(mp->window[i]);
    a.x = static_cast<T *>(x);
    a.s = static_cast<T *>(s);
    a.u = static_cast<T *>(u);
    a.s_ref = static_cast<T *>(s_ref);
    a.y = static_cast<T *>(y);
    a.zeta = static_cast<T *>(zeta);
    a.xi = static_cast<T *>(xi);
    a.P = sc->P;
    a.FR = sc->FR;
    a.FO = sc->FO;
    a.mask = sc->d_mask;
    a.x_hist = static_cast<T *>(x_hist);
    a.u_hist = static_cast<T *>(u_hist);
    a.n_steps = mp->n_steps;
    a.collided = collided;
    a.iters_hist = iters_hist;
    a.iters = sc->d_mpc_i;
    oca_admm_report rep;
    rep.iters = sc->d_mpc_i;
    rep.status = sc->d_mpc_i + sc->S;
    T *rf = reinterpret_cast<T *>(sc->d_mpc_f);
    rep.r_pri = rf;
    rep.r_dual = rf + sc->S;
    rep.cost = rf + 2 * sc->S;
    int max_blk = 1;
    for (const ScenMeta &m2 : sc->meta) max_blk = std::max(max_blk, m2.M * m2.NP);
    OCA_CK(cudaMemsetAsync(collided, 0xff, sizeof(int32_t) * sc->S, st));
    cudaGraphExec_t graph = nullptr;  // the iteration graph, the same for every control step
    oca_status out = OCA_OK;
    for (int c = 0; c < mp->n_steps && out == OCA_OK; ++c) {
        a.c = c;
        if (launch_mpc<T>(a, 0, sc->S, max_blk, st) != cudaSuccess ||
            (c > 0 && launch_mpc<T>(a, 1, sc->S, max_blk, st) != cudaSuccess)) {
            out = OCA_ERR_CUDA;
            break;
        }
        out = admm_impl<T>(sc, m, pr, s_ref, s, u, y, zeta, xi, &rep, st, nullptr, sc->d_mask, &graph, false);
        if (out == OCA_OK && (launch_mpc<T>(a, 2, sc->S, max_blk, st) != cudaSuccess ||
                              launch_mpc<T>(a, 3, sc->S, max_blk, st) != cudaSuccess))
            out = OCA_ERR_CUDA;
    }
    if (graph) cudaGraphExecDestroy(graph);
    return out;
}

void free_scene(oca_scene *sc) {
    if (!sc) return;
    cudaFree(sc->d_meta);
    cudaFree(sc->d_tiles);
    cudaFree(sc->d_obs_nf);
    cudaFree(sc->d_part_nf);
    cudaFree(sc->d_part_link);
    cudaFree(sc->d_part_radius);
    cudaFree(sc->d_pose);
    cudaFree(sc->d_stats);
    cudaFree(sc->d_y2);
    cudaFree(sc->d_ric);
    cudaFree(sc->d_res);
    cudaFree(sc->d_ric_off);
    cudaFree(sc->d_status);
    cudaFree(sc->d_mpc_i);
    cudaFree(sc->d_rev_iters);
    cudaFree(sc->d_mpc_f);
    cudaFree(sc->d_mask);
    cudaFree(sc->d_iter);
    cudaFree(sc->d_active);
    cudaFree(sc->d_err);
    cudaFree(sc->d_box);
    cudaFree(sc->d_box_res);
    if (sc->h_active) cudaFreeHost(sc->h_active);
    delete sc;
}

template <typename P>
oca_status dmalloc(P **p, size_t bytes) {
    if (cudaMalloc(reinterpret_cast<void **>(p), bytes ? bytes : 16) != cudaSuccess) return OCA_ERR_NO_MEMORY;
    return OCA_OK;
}

}  // namespace

extern "C" {

const char *oca_status_string(oca_status st) {
    switch (st) {
        case OCA_OK: return "OCA_OK";
        case OCA_ERR_INVALID_ARGUMENT: return "OCA_ERR_INVALID_ARGUMENT";
        case OCA_ERR_CUDA: return "OCA_ERR_CUDA";
        case OCA_ERR_NO_MEMORY: return "OCA_ERR_NO_MEMORY";
        case OCA_ERR_UNSUPPORTED: return "OCA_ERR_UNSUPPORTED";
        case OCA_ERR_CAPACITY: return "OCA_ERR_CAPACITY";
    }
    return "OCA_ERR_UNKNOWN";
}

oca_status oca_create(oca_ctx **out, int device) {
    if (!out) return OCA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) return OCA_ERR_CUDA;
    if (device < 0 || device >= n) return OCA_ERR_INVALID_ARGUMENT;
    if (cudaSetDevice(device) != cudaSuccess) return OCA_ERR_CUDA;
    oca_ctx *c = new (std::nothrow) oca_ctx;
    if (!c) return OCA_ERR_NO_MEMORY;
    c->device = device;
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
        delete c;
        return OCA_ERR_CUDA;
    }
    *out = c;
    return OCA_OK;
}

void oca_destroy(oca_ctx *ctx) {
    if (!ctx) return;
    for (auto &row : ctx->ev)
        for (auto &e : row)
            if (e) cudaEventDestroy(e);
    delete ctx;
}

oca_status oca_profile_enable(oca_ctx *ctx, int enable) {
    if (!ctx) return OCA_ERR_INVALID_ARGUMENT;
    if (enable) {
        for (auto &row : ctx->ev)
            for (auto &e : row)
                if (!e && cudaEventCreate(&e) != cudaSuccess) return OCA_ERR_CUDA;
        ctx->pair_ms = ctx->traj_ms = 0;
        ctx->pair_launches = ctx->traj_launches = 0;
    }
    ctx->prof = enable != 0;
    return OCA_OK;
}

oca_status oca_profile_read(const oca_ctx *ctx, oca_profile_stats *out) {
    if (!ctx || !out) return OCA_ERR_INVALID_ARGUMENT;
    out->pair_ms = ctx->pair_ms;
    out->traj_ms = ctx->traj_ms;
    out->pair_launches = ctx->pair_launches;
    out->traj_launches = ctx->traj_launches;
    return OCA_OK;
}

oca_status oca_scene_create(oca_ctx *ctx, const oca_scene_desc *d, oca_scene **out) {
    if (!ctx || !d || !out) return OCA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    if (d->dim != 2 && d->dim != 3) return OCA_ERR_INVALID_ARGUMENT;
    if (d->dtype != OCA_F32 && d->dtype != OCA_F64) return OCA_ERR_INVALID_ARGUMENT;
    if (d->n_scen < 1 || d->n_scen > 65535) return d->n_scen < 1 ? OCA_ERR_INVALID_ARGUMENT : OCA_ERR_CAPACITY;
    if (d->fo_max < 1 || d->fr_max < 1) return OCA_ERR_INVALID_ARGUMENT;
    if (d->fo_max > OCA_MAX_OBS_FACES || d->fr_max > OCA_MAX_PART_FACES) return OCA_ERR_CAPACITY;
    if (!d->obs_begin || !d->obs_nf || !d->part_begin || !d->part_nf || !d->part_link || !d->horizon)
        return OCA_ERR_INVALID_ARGUMENT;
    if (!d->obs_C || !d->obs_d || !d->part_A || !d->part_b || !d->part_off) return OCA_ERR_INVALID_ARGUMENT;
    const int S = d->n_scen;
    if (d->obs_begin[0] != 0 || d->part_begin[0] != 0) return OCA_ERR_INVALID_ARGUMENT;
    for (int s = 0; s < S; ++s) {
        if (d->obs_begin[s + 1] < d->obs_begin[s] + 1) return OCA_ERR_INVALID_ARGUMENT;  // >= 1 obstacle
        if (d->part_begin[s + 1] < d->part_begin[s] + 1) return OCA_ERR_INVALID_ARGUMENT; // >= 1 part
        if (d->horizon[s] < 1) return OCA_ERR_INVALID_ARGUMENT;
        if (d->horizon[s] > OCA_MAX_HORIZON) return OCA_ERR_CAPACITY;
    }
    const int M_tot = d->obs_begin[S], P_tot = d->part_begin[S];
    for (int i = 0; i < M_tot; ++i)
        if (d->obs_nf[i] < 1 || d->obs_nf[i] > d->fo_max) return OCA_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < P_tot; ++i) {
        if (d->part_nf[i] < d->dim + 1 || d->part_nf[i] > d->fr_max) return OCA_ERR_INVALID_ARGUMENT;
        if (d->part_link[i] < 0 || d->part_link[i] > 1 || (d->dim == 3 && d->part_link[i] != 0))
            return OCA_ERR_INVALID_ARGUMENT;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return OCA_ERR_CUDA;
    oca_scene *sc = new (std::nothrow) oca_scene;
    if (!sc) return OCA_ERR_NO_MEMORY;
    sc->ctx = ctx;
    sc->dim = d->dim;
    sc->dtype = d->dtype;
    sc->S = S;
    sc->FO = d->fo_max;
    sc->FR = d->fr_max;
    sc->M_tot = M_tot;
    sc->P_tot = P_tot;
    sc->obs_C = d->obs_C;
    sc->obs_d = d->obs_d;
    sc->part_A = d->part_A;
    sc->part_b = d->part_b;
    sc->part_off = d->part_off;
    sc->ny_max = d->fr_max + d->fo_max + 1;
    sc->ns_max = d->dim == 3 ? 12 : 5;
    sc->nu_max = d->dim == 3 ? 4 : 2;
    sc->meta.resize(S);
    sc->pair_begin.assign(S + 1, 0);
    sc->state_begin.assign(S + 1, 0);
    sc->ctrl_begin.assign(S + 1, 0);
    long long qtot = 0, tiles = 0;
    std::vector<long long> cost(S);
    std::vector<int> Ms;
    for (int s = 0; s < S; ++s) {
        ScenMeta &m = sc->meta[s];
        m.N = d->horizon[s];
        m.M = d->obs_begin[s + 1] - d->obs_begin[s];
        m.NP = d->part_begin[s + 1] - d->part_begin[s];
        m.obs0 = d->obs_begin[s];
        m.part0 = d->part_begin[s];
        m.qbeg = (int)qtot;
        m.state0 = (int)sc->state_begin[s];
        m.ctrl0 = (int)sc->ctrl_begin[s];
        m.tile0 = (int)tiles;
        const int Q = m.NP * m.N;
        m.ntile = (Q + 31) / 32;
        m.pair0 = sc->pair_begin[s];
        sc->pair_begin[s + 1] = sc->pair_begin[s] + (long long)m.M * Q;
        sc->state_begin[s + 1] = sc->state_begin[s] + m.N + 1;
        sc->ctrl_begin[s + 1] = sc->ctrl_begin[s] + m.N;
        qtot += Q;
        tiles += m.ntile;
        sc->maxQ = std::max(sc->maxQ, Q);
        sc->maxN = std::max(sc->maxN, m.N);
        long long faces = 0;
        for (int j = 0; j < m.M; ++j) faces += d->obs_nf[m.obs0 + j] + 1;
        cost[s] = faces;
        Ms.push_back(m.M);
    }
    if (qtot > (1LL << 30) || tiles > (1LL << 30) || sc->state_begin[S] > (1LL << 30)) {
        free_scene(sc);
        return OCA_ERR_CAPACITY;
    }
    sc->P = sc->pair_begin[S];
    sc->n_states = sc->state_begin[S];
    sc->n_ctrls = sc->ctrl_begin[S];
    sc->Qtot = (int)qtot;
    sc->n_tiles = (int)tiles;
    // tiles in descending cost order (heaviest scenarios first)
    std::vector<Tile> tl;
    tl.reserve(tiles);
    std::vector<int> order(S);
    for (int s = 0; s < S; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    for (int s : order)
        for (int k = 0; k < sc->meta[s].ntile; ++k) {
            const int cols = sc->meta[s].NP * sc->meta[s].N - 32 * k;
            tl.push_back(Tile{s, 32 * k, cols <= 16 ? 1 : 0});
        }
    // warps per tile: about 8 obstacles per warp at the median obstacle count
    std::nth_element(Ms.begin(), Ms.begin() + Ms.size() / 2, Ms.end());
    const int Mmed = Ms[Ms.size() / 2];
    sc->W = std::max(1, std::min(16, (Mmed + 7) / 8));
    while (sc->W > 1 && !warps_fit(sc, sc->W)) --sc->W;

    const size_t ts = dsize(d->dtype);
    const int PK = d->dim + d->dim * d->dim;
    const int NSTAT = d->dim * (d->dim + 1) / 2 + d->dim + d->dim * d->dim;
    oca_status e = OCA_OK;
    std::vector<long long> roff(S);
    long long rtot = 0;
    const int rkind = d->dim == 3 ? 2 : 1;
    for (int s = 0; s < S; ++s) {
        roff[s] = rtot;
        rtot += riccati_scratch_elems(rkind, sc->meta[s].N);
        rtot = (rtot + 3) & ~3LL;
    }
    if ((e = dmalloc(&sc->d_meta, sizeof(ScenMeta) * S)) != OCA_OK ||
        (e = dmalloc(&sc->d_tiles, sizeof(Tile) * tl.size())) != OCA_OK ||
        (e = dmalloc(&sc->d_obs_nf, sizeof(int) * M_tot)) != OCA_OK ||
        (e = dmalloc(&sc->d_part_nf, sizeof(int) * P_tot)) != OCA_OK ||
        (e = dmalloc(&sc->d_part_link, sizeof(int) * P_tot)) != OCA_OK ||
        (e = dmalloc(&sc->d_part_radius, sizeof(double) * P_tot)) != OCA_OK ||
        (e = dmalloc(&sc->d_pose, ts * PK * (size_t)qtot)) != OCA_OK ||
        (e = dmalloc(&sc->d_stats, ts * NSTAT * (size_t)qtot)) != OCA_OK ||
        (e = dmalloc(&sc->d_y2, ts * sc->ny_max * (size_t)sc->P)) != OCA_OK ||
        (e = dmalloc(&sc->d_ric, sizeof(double) * (size_t)rtot)) != OCA_OK ||
        (e = dmalloc(&sc->d_ric_off, sizeof(long long) * S)) != OCA_OK ||
        (e = dmalloc(&sc->d_res, sizeof(double) * 4 * (size_t)tiles)) != OCA_OK ||
        (e = dmalloc(&sc->d_status, sizeof(int) * S)) != OCA_OK ||
        (e = dmalloc(&sc->d_mpc_i, sizeof(int) * 2 * S)) != OCA_OK ||
        (e = dmalloc(&sc->d_rev_iters, sizeof(int) * S)) != OCA_OK ||
        (e = dmalloc(&sc->d_mpc_f, sizeof(double) * 3 * S)) != OCA_OK ||
        (e = dmalloc(&sc->d_mask, (size_t)M_tot)) != OCA_OK ||
        (e = dmalloc(&sc->d_iter, sizeof(int))) != OCA_OK ||
        (e = dmalloc(&sc->d_active, sizeof(int))) != OCA_OK ||
        (e = dmalloc(&sc->d_err, sizeof(int))) != OCA_OK ||
        (e = dmalloc(&sc->d_box, ts * 2 * ((size_t)sc->n_states * sc->ns_max + (size_t)sc->n_ctrls * sc->nu_max))) != OCA_OK ||
        (e = dmalloc(&sc->d_box_res, sizeof(double) * 2 * (size_t)S)) != OCA_OK) {
        free_scene(sc);
        return e;
    }
    if (cudaMallocHost(reinterpret_cast<void **>(&sc->h_active), sizeof(int)) != cudaSuccess) {
        sc->h_active = nullptr;
        free_scene(sc);
        return OCA_ERR_NO_MEMORY;
    }
    bool ok = cudaMemcpy(sc->d_meta, sc->meta.data(), sizeof(ScenMeta) * S, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(sc->d_tiles, tl.data(), sizeof(Tile) * tl.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(sc->d_obs_nf, d->obs_nf, sizeof(int) * M_tot, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(sc->d_part_nf, d->part_nf, sizeof(int) * P_tot, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(sc->d_part_link, d->part_link, sizeof(int) * P_tot, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(sc->d_ric_off, roff.data(), sizeof(long long) * S, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemset(sc->d_err, 0, sizeof(int)) == cudaSuccess &&
              cudaMemset(sc->d_res, 0, sizeof(double) * 4 * (size_t)tiles) == cudaSuccess;
    if (!ok) {
        free_scene(sc);
        return OCA_ERR_CUDA;
    }
    const int nthr = std::max(M_tot, P_tot);
    if (d->dtype == OCA_F32)
        k_validate<float><<<(nthr + 127) / 128, 128>>>(
            static_cast<const float *>(d->obs_C), static_cast<const float *>(d->obs_d), sc->d_obs_nf, M_tot,
            static_cast<const float *>(d->part_A), static_cast<const float *>(d->part_b), sc->d_part_nf, P_tot,
            static_cast<const float *>(d->part_off), d->fo_max, d->fr_max, d->dim, sc->d_part_radius, sc->d_err);
    else
        k_validate<double><<<(nthr + 127) / 128, 128>>>(
            static_cast<const double *>(d->obs_C), static_cast<const double *>(d->obs_d), sc->d_obs_nf, M_tot,
            static_cast<const double *>(d->part_A), static_cast<const double *>(d->part_b), sc->d_part_nf, P_tot,
            static_cast<const double *>(d->part_off), d->fo_max, d->fr_max, d->dim, sc->d_part_radius, sc->d_err);
    int herr = 0;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&herr, sc->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        free_scene(sc);
        return OCA_ERR_CUDA;
    }
    if (herr) {
        free_scene(sc);
        return OCA_ERR_INVALID_ARGUMENT;
    }
    *out = sc;
    return OCA_OK;
}

void oca_scene_destroy(oca_scene *scene) { free_scene(scene); }

oca_status oca_scene_info_get(const oca_scene *sc, oca_scene_info *info) {
    if (!sc || !info) return OCA_ERR_INVALID_ARGUMENT;
    info->n_pairs = sc->P;
    info->n_states = sc->n_states;
    info->n_ctrls = sc->n_ctrls;
    info->ny_max = sc->ny_max;
    info->n_tiles = sc->n_tiles;
    info->pair_begin = sc->pair_begin.data();
    info->state_begin = sc->state_begin.data();
    info->ctrl_begin = sc->ctrl_begin.data();
    return OCA_OK;
}

oca_status oca_scene_set_warps(oca_scene *sc, int warps) {
    if (!sc || warps < 1 || warps > 16) return OCA_ERR_INVALID_ARGUMENT;
    if (!warps_fit(sc, warps)) return OCA_ERR_CAPACITY;
    sc->W = warps;
    return OCA_OK;
}

int oca_scene_get_warps(const oca_scene *sc) { return sc ? sc->W : -1; }

oca_status oca_scale_detect_batch(oca_ctx *ctx, const oca_scene *scene, const oca_model *model, const void *states,
                                  void *alpha, void *lambda, void *mu, double *margin, int32_t *verdict,
                                  int32_t *status, void *stream) {
    if (!ctx || !scene || !states || !alpha) return OCA_ERR_INVALID_ARGUMENT;
    oca_scene *sc = const_cast<oca_scene *>(scene);
    oca_status e = check_model(sc, model);
    if (e != OCA_OK) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (sc->dtype == OCA_F32)
        return scale_impl<float>(sc, model, states, alpha, lambda, mu, margin, verdict, status, st);
    return scale_impl<double>(sc, model, states, alpha, lambda, mu, margin, verdict, status, st);
}

oca_status oca_cert_margin_batch(oca_ctx *ctx, const oca_scene *scene, const oca_model *model, const void *states,
                                 const void *lambda, const void *mu, double *margin, void *stream) {
    if (!ctx || !scene || !states || !lambda || !mu || !margin) return OCA_ERR_INVALID_ARGUMENT;
    oca_scene *sc = const_cast<oca_scene *>(scene);
    oca_status e = check_model(sc, model);
    if (e != OCA_OK) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (sc->dtype == OCA_F32) return cert_impl<float>(sc, model, states, lambda, mu, margin, st);
    return cert_impl<double>(sc, model, states, lambda, mu, margin, st);
}

oca_status oca_pair_qp_batch(oca_ctx *ctx, const oca_scene *scene, const oca_model *model, const void *states,
                             const void *zeta, const void *xi, double prox, const void *y_in, void *y_out,
                             void *v_out, void *obj_out, int32_t *status_out, void *stream) {
    if (!ctx || !scene || !states || !zeta || !xi || !y_in || !y_out) return OCA_ERR_INVALID_ARGUMENT;
    if (!(prox >= 0.0) || !std::isfinite(prox)) return OCA_ERR_INVALID_ARGUMENT;
    oca_scene *sc = const_cast<oca_scene *>(scene);
    oca_status e = check_model(sc, model);
    if (e != OCA_OK) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (sc->dtype == OCA_F32)
        return pairqp_impl<float>(sc, model, states, zeta, xi, prox, y_in, y_out, v_out, obj_out, status_out, st);
    return pairqp_impl<double>(sc, model, states, zeta, xi, prox, y_in, y_out, v_out, obj_out, status_out, st);
}

oca_status oca_admm_solve(oca_ctx *ctx, const oca_scene *scene, const oca_model *model,
                          const oca_admm_params *params, const void *s_ref, void *s, void *u, void *y, void *zeta,
                          void *xi, const oca_admm_report *report, void *stream) {
    if (!ctx || !scene || !params || !s_ref || !s || !u || !y || !zeta || !xi || !report) return OCA_ERR_INVALID_ARGUMENT;
    if (!report->iters || !report->status || !report->r_pri || !report->r_dual || !report->cost)
        return OCA_ERR_INVALID_ARGUMENT;
    if (!(params->sigma > 0.0) || !(params->prox >= 0.0) || !(params->eps_pri >= 0.0) || !(params->eps_dual >= 0.0) ||
        params->max_iter < 0 || !std::isfinite(params->sigma) || !std::isfinite(params->prox) ||
        !(params->rho_box >= 0.0) || !(params->damp >= 0.0) || !std::isfinite(params->rho_box) ||
        !std::isfinite(params->damp))
        return OCA_ERR_INVALID_ARGUMENT;
    oca_scene *sc = const_cast<oca_scene *>(scene);
    oca_status e = check_model(sc, model);
    if (e != OCA_OK) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (sc->dtype == OCA_F32) return admm_impl<float>(sc, model, params, s_ref, s, u, y, zeta, xi, report, st);
    return admm_impl<double>(sc, model, params, s_ref, s, u, y, zeta, xi, report, st);
}


oca_status oca_admm_tape_bytes(const oca_scene *scene, const oca_model *model, int32_t max_iter, int64_t *bytes) {
    if (!scene || !bytes || max_iter < 0) return OCA_ERR_INVALID_ARGUMENT;
    oca_status e = check_model(scene, model);
    if (e != OCA_OK) return e;
    *bytes = (int64_t)tape_layout(scene, model->kind, max_iter).bytes;
    return OCA_OK;
}

oca_status oca_admm_fixed_point_tape_bytes(const oca_scene *scene, const oca_model *model, int64_t *bytes) {
    if (!scene || !bytes) return OCA_ERR_INVALID_ARGUMENT;
    oca_status e = check_model(scene, model);
    if (e != OCA_OK) return e;
    *bytes = (int64_t)tape_layout(scene, model->kind, 0, true).bytes;
    return OCA_OK;
}

static oca_status check_admm_args(const oca_ctx *ctx, const oca_scene *scene, const oca_admm_params *params,
                                  const void *s_ref, const void *s, const void *u, const void *y, const void *zeta,
                                  const void *xi, const oca_admm_report *report) {
    if (!ctx || !scene || !params || !s_ref || !s || !u || !y || !zeta || !xi || !report) return OCA_ERR_INVALID_ARGUMENT;
    if (!report->iters || !report->status || !report->r_pri || !report->r_dual || !report->cost)
        return OCA_ERR_INVALID_ARGUMENT;
    if (!(params->sigma > 0.0) || !(params->prox >= 0.0) || !(params->eps_pri >= 0.0) || !(params->eps_dual >= 0.0) ||
        params->max_iter < 0 || !std::isfinite(params->sigma) || !std::isfinite(params->prox) ||
        !(params->rho_box >= 0.0) || !(params->damp >= 0.0) || !std::isfinite(params->rho_box) ||
        !std::isfinite(params->damp))
        return OCA_ERR_INVALID_ARGUMENT;
    return OCA_OK;
}

oca_status oca_admm_solve_taped(oca_ctx *ctx, const oca_scene *scene, const oca_model *model,
                                const oca_admm_params *params, const void *s_ref, void *s, void *u, void *y,
                                void *zeta, void *xi, const oca_admm_report *report, void *tape, int64_t tape_bytes,
                                void *stream) {
    oca_status e = check_admm_args(ctx, scene, params, s_ref, s, u, y, zeta, xi, report);
    if (e != OCA_OK) return e;
    oca_scene *sc = const_cast<oca_scene *>(scene);
    if ((e = check_model(sc, model)) != OCA_OK) return e;
    if (!tape || reinterpret_cast<uintptr_t>(tape) % 256 != 0) return OCA_ERR_INVALID_ARGUMENT;
    const bool fp = (params->flags & OCA_ADMM_FIXED_POINT) != 0;
    if (tape_bytes < (int64_t)tape_layout(sc, model->kind, params->max_iter, fp).bytes) return OCA_ERR_CAPACITY;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (sc->dtype == OCA_F32) return admm_impl<float>(sc, model, params, s_ref, s, u, y, zeta, xi, report, st, tape);
    return admm_impl<double>(sc, model, params, s_ref, s, u, y, zeta, xi, report, st, tape);
}

oca_status oca_admm_backward(oca_ctx *ctx, const oca_scene *scene, const oca_model *model,
                             const oca_admm_params *params, const void *s_ref, void *tape, int64_t tape_bytes,
                             const int32_t *iters, const void *grad_cost, const void *grad_alpha,
                             void *grad_obs_offset, void *grad_obs_center, void *grad_state0, void *stream) {
    if (!ctx || !scene || !params || !s_ref || !tape || !iters || !grad_cost) return OCA_ERR_INVALID_ARGUMENT;
    if (!grad_obs_offset && !grad_obs_center && !grad_state0) return OCA_ERR_INVALID_ARGUMENT;
    if (reinterpret_cast<uintptr_t>(tape) % 256 != 0 || params->max_iter < 0) return OCA_ERR_INVALID_ARGUMENT;
    if (!(params->sigma > 0.0) || !(params->rho_box >= 0.0) || !(params->damp >= 0.0)) return OCA_ERR_INVALID_ARGUMENT;
    if (!(params->prox > 0.0)) return OCA_ERR_UNSUPPORTED;
    oca_scene *sc = const_cast<oca_scene *>(scene);
    oca_status e = check_model(sc, model);
    if (e != OCA_OK) return e;
    const bool fp = (params->flags & OCA_ADMM_FIXED_POINT) != 0;
    if (tape_bytes < (int64_t)tape_layout(sc, model->kind, params->max_iter, fp).bytes) return OCA_ERR_CAPACITY;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (sc->dtype == OCA_F32)
        return backward_impl<float>(sc, model, params, s_ref, tape, iters, grad_cost, grad_alpha, grad_obs_offset,
                                    grad_obs_center, grad_state0, st);
    return backward_impl<double>(sc, model, params, s_ref, tape, iters, grad_cost, grad_alpha, grad_obs_offset,
                                 grad_obs_center, grad_state0, st);
}


oca_status oca_mpc_run(oca_ctx *ctx, const oca_scene *scene, const oca_model *model, const oca_admm_params *params,
                       const oca_mpc_params *mpc, const void *ref, int32_t T_ref, const void *obs_center, void *x,
                       void *s_ref, void *s, void *u, void *y, void *zeta, void *xi, void *x_hist, void *u_hist,
                       int32_t *iters_hist, int32_t *collided, void *stream) {
    if (!ctx || !scene || !params || !mpc || !ref || !obs_center || !x || !s_ref || !s || !u || !y || !zeta || !xi ||
        !x_hist || !u_hist || !iters_hist || !collided)
        return OCA_ERR_INVALID_ARGUMENT;
    if (!(params->sigma > 0.0) || !(params->prox >= 0.0) || !(params->eps_pri >= 0.0) || !(params->eps_dual >= 0.0) ||
        params->max_iter < 0 || !(params->rho_box >= 0.0) || !(params->damp >= 0.0))
        return OCA_ERR_INVALID_ARGUMENT;
    if (mpc->n_steps < 1 || T_ref < 1) return OCA_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < 3; ++i)
        if (std::isnan(mpc->window[i])) return OCA_ERR_INVALID_ARGUMENT;
    oca_scene *sc = const_cast<oca_scene *>(scene);
    const oca_status e = check_model(sc, model);
    if (e != OCA_OK) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (sc->dtype == OCA_F32)
        return mpc_impl<float>(sc, model, params, mpc, ref, T_ref, obs_center, x, s_ref, s, u, y, zeta, xi, x_hist,
                               u_hist, iters_hist, collided, st);
    return mpc_impl<double>(sc, model, params, mpc, ref, T_ref, obs_center, x, s_ref, s, u, y, zeta, xi, x_hist,
                            u_hist, iters_hist, collided, st);
}


oca_status oca_pair_qp_lemke_batch(oca_ctx *ctx, const oca_scene *scene, const oca_model *model, const void *states,
                                   const void *zeta, const void *xi, double prox, const void *y_in, void *y_out,
                                   void *v_out, void *obj_out, int32_t *status_out, void *stream) {
    if (!ctx || !scene || !states || !zeta || !xi || !y_in || !y_out || !(prox >= 0.0) || !std::isfinite(prox))
        return OCA_ERR_INVALID_ARGUMENT;
    oca_scene *sc = const_cast<oca_scene *>(scene);
    const oca_status e = check_model(sc, model);
    if (e != OCA_OK) return e;
    if (y_out == y_in) return OCA_ERR_INVALID_ARGUMENT;
    if (sc->FR + sc->FO + 1 > 32) return OCA_ERR_UNSUPPORTED;  // one lane per LCP row
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (sc->dtype == OCA_F32)
        return lemke_impl<float>(sc, model, states, zeta, xi, prox, y_in, y_out, v_out, obj_out, status_out, st);
    return lemke_impl<double>(sc, model, states, zeta, xi, prox, y_in, y_out, v_out, obj_out, status_out, st);
}

}  // extern "C"
