// Internal definitions shared by the CUDA translation units of liboca.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "oca.h"

namespace oca {

constexpr int kMaxFO = OCA_MAX_OBS_FACES;
constexpr int kMaxFR = OCA_MAX_PART_FACES;
constexpr int kActive = OCA_SCEN_ACTIVE;

// Per-scenario metadata on the device.
struct ScenMeta {
    int N;       // horizon N_s (constraint steps t = 1..N)
    int M;       // obstacles
    int NP;      // robot parts
    int obs0;    // first obstacle (global index)
    int part0;   // first part (global index)
    int qbeg;    // first (part, t) lane index; Q_s = NP * N lanes
    int state0;  // first state row
    int ctrl0;   // first control row
    int tile0;   // first work tile (natural order)
    int ntile;   // ceil(Q_s / 32)
    long long pair0;  // first pair
};

// A work tile: 32 consecutive (part, t) lanes of one scenario.
struct Tile {
    int scen;
    int q0;
    int split;  // a scenario's last tile with <= 16 columns: the pair kernel runs it as half-warps
};

// Scene geometry as kernels see it.
template <typename T>
struct Geom {
    const T *obs_C;    // [M_tot][FO][D]
    const T *obs_d;    // [M_tot][FO]
    const int *obs_nf; // [M_tot]
    const T *part_A;   // [P_tot][FR][D]
    const T *part_b;   // [P_tot][FR]
    const int *part_nf;
    const int *part_link;
    const T *part_off; // [P_tot][D]
    int FO, FR;
};

template <typename T>
struct DevModel {
    int kind;
    T dt;
    T p[8];
    T Qs[12];
    T Qu[4];
    T s_lo[12], s_hi[12];  // state box (|bound| >= 1e29: none)
    T u_lo[4], u_hi[4];    // control box
};

template <int KIND> struct MDims;
template <> struct MDims<0> { enum { NS = 4, NU = 2, D = 2, NROT = 1 }; };
template <> struct MDims<1> { enum { NS = 5, NU = 2, D = 2, NROT = 1 }; };
template <> struct MDims<2> { enum { NS = 12, NU = 4, D = 3, NROT = 3 }; };

// pose record per (scenario, part, t): rho (D) then R (D*D, row-major)
template <int D> struct PoseDims { enum { PK = D + D * D }; };
// Gauss-Newton statistics per (scenario, part, t): W = sum w w^T (sym, D(D+1)/2),
// Wc = sum c w (D), E = sum w e^T (D*D)
template <int D> struct StatDims { enum { NW = D * (D + 1) / 2, NSTAT = D * (D + 1) / 2 + D + D * D }; };

#define OCA_HD __host__ __device__

// ---- math overloads --------------------------------------------------------
OCA_HD inline float m_sin(float x) { return sinf(x); }
OCA_HD inline double m_sin(double x) { return sin(x); }
OCA_HD inline float m_cos(float x) { return cosf(x); }
OCA_HD inline double m_cos(double x) { return cos(x); }
OCA_HD inline float m_tan(float x) { return tanf(x); }
OCA_HD inline double m_tan(double x) { return tan(x); }
OCA_HD inline float m_sqrt(float x) { return sqrtf(x); }
OCA_HD inline double m_sqrt(double x) { return sqrt(x); }
// 1 / sqrt(x): the hardware-approximated reciprocal square root on the device
// (within a few ulp; used where only a search direction depends on it)
OCA_HD inline float m_rsqrt(float x) {
#ifdef __CUDA_ARCH__
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}
OCA_HD inline double m_rsqrt(double x) {
#ifdef __CUDA_ARCH__
    return rsqrt(x);
#else
    return 1.0 / sqrt(x);
#endif
}
// 1 / x for a positive normal x: in FP32 on the device the hardware
// approximation of the reciprocal (about 1 ulp; used for metric weights, where
// any positive value gives a valid method and the solve uses the same value
// throughout), otherwise the IEEE division
OCA_HD inline float m_rcp(float x) {
#ifdef __CUDA_ARCH__
    return __fdividef(1.0f, x);
#else
    return 1.0f / x;
#endif
}
OCA_HD inline double m_rcp(double x) { return 1.0 / x; }
OCA_HD inline float m_abs(float x) { return fabsf(x); }
OCA_HD inline double m_abs(double x) { return fabs(x); }
template <typename T> OCA_HD inline T m_eps();
template <> OCA_HD inline float m_eps<float>() { return 1.1920929e-7f; }
template <> OCA_HD inline double m_eps<double>() { return 2.220446049250313e-16; }
OCA_HD inline bool m_finite(float x) { return isfinite(x); }
OCA_HD inline bool m_finite(double x) { return isfinite(x); }

template <typename T>
OCA_HD inline T ldg(const T *p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

#ifdef __CUDACC__
// Asynchronous global -> shared copy of one element (cp.async, 4 or 8 bytes,
// both addresses aligned to the element size), its group commit and the wait
// for every group this thread committed.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
#endif

// ---- kernel argument blocks -------------------------------------------------
template <typename T>
struct PoseArgs {
    const ScenMeta *meta;
    int n_scen;
    Geom<T> g;
    DevModel<T> model;
    const T *states;   // [n_states][NS]
    T *pose;           // [PK][Qtot]
    int Qtot;
    const int *scen_status;  // may be null: then every scenario is posed
};

template <typename T>
struct PairArgs {
    const ScenMeta *meta;
    const Tile *tiles;      // launch order (cost-sorted)
    Geom<T> g;
    const T *pose;          // [PK][Qtot]
    int Qtot;
    long long P;            // total pairs (component stride)
    T *zeta;                // [P]
    T *xi;                  // [D][P]
    const T *y_in;          // [NY][P]
    T *y_out;               // [NY][P]
    T *v_out;               // [D+1][P] or null
    T *obj_out;             // [P] or null
    int *status_out;        // [P] or null
    T *stats;               // [NSTAT][Qtot] (ADMM mode)
    double *res;            // [2][n_tiles][2] residual partials (ADMM mode)
    int n_tiles;
    const int *scen_status; // ADMM mode
    const int *iter;        // ADMM mode: device iteration counter j
    int max_iter;
    T prox;
    const unsigned char *obs_mask;  // [M_tot] or null: obstacles with 0 are skipped (their y passed through)
};

template <typename T>
struct ScaleArgs {
    const ScenMeta *meta;
    const Tile *tiles;
    Geom<T> g;
    const T *pose;
    int Qtot;
    long long P;
    const double *part_radius;  // [P_tot] largest vertex norm of each part
    T *alpha;
    T *lambda;      // [FR][P] or null
    T *mu;          // [FO][P] or null
    double *margin; // [P] or null
    int *verdict;   // [P] or null
    int *status;    // [P] or null
};

// FP64 certificate margin of caller-given dual variables (oca_cert_margin_batch)
template <typename T>
struct CertArgs {
    const ScenMeta *meta;
    const Tile *tiles;
    Geom<T> g;
    DevModel<double> model;     // poses are formed in FP64 from the stored states
    const T *states;            // [n_states][NS]
    long long P;
    const double *part_radius;  // [P_tot]
    const T *lambda;            // [FR][P]
    const T *mu;                // [FO][P]
    double *margin;             // [P]
};

template <typename T>
struct RicArgs {
    const ScenMeta *meta;
    int n_scen;
    Geom<T> g;
    DevModel<T> model;
    T sigma, eps_pri, eps_dual, rho_box, damp;
    T *box_zs, *box_ws;  // [n_states][NS] bounded copy and scaled dual of the states
    T *box_zu, *box_wu;  // [n_ctrls][NU]
    double *box_res;     // [S][2] box residuals of the last trajectory step
    int max_iter;
    const int *iter;
    const T *s_ref;
    T *s;
    T *u;
    T *pose;
    const T *stats;
    int Qtot;
    const double *res;  // [2][n_tiles][2]
    int n_tiles;
    int *scen_status;
    int *status_out;
    int *iters_out;
    T *r_pri_out, *r_dual_out, *cost_out;
    int *active_count;
    void *scratch;      // per-stage workspace (factorisation precision)
    const long long *scratch0;  // per-scenario offset into scratch (elements)
};

// ---- adjoint (oca_admm_backward) --------------------------------------------
// Slots of a taped solve: iterate k of every array lives at base + k * slot.
template <typename T>
struct TapeView {
    const T *y;      // y^k, k = 0..K            [NY][P] per slot
    const T *zx;     // (zeta^k, xi^k) after the head of iteration k, k = 0..K-1  [1+D][P]
    const T *stats;  // Gauss-Newton statistics of iteration k  [NSTAT][Qtot]
    const T *s, *u;  // s^k, u^k, k = 0..K      [n_states][NS], [n_ctrls][NU]
    const T *box;    // z_s, w_s, z_u, w_u after the box update giving iterate k
    long long y_slot, zx_slot, stats_slot, s_slot, u_slot, box_slot;
    long long n_states, n_ctrls;  // row counts (box sub-array offsets)
};

template <typename T>
struct AdjTrajArgs {
    const ScenMeta *meta;
    Geom<T> g;
    DevModel<T> model;
    T sigma, rho_box, damp;
    const T *s_ref;
    int Qtot;
    const int *iters;       // [S] iterations of the taped solve
    int k;                  // reverse step: iteration k is differentiated
    TapeView<T> tape;
    const T *grad_cost;     // [S] (seed only)
    T *sb, *ub;             // adjoints of s, u (rows as the state arrays)
    T *zsb, *wsb, *zub, *wub;  // adjoints of the box block
    T *statsb;              // [NSTAT][Qtot] adjoint of the statistics of iteration k (out)
    const T *poseb;         // [PK][Qtot] adjoint of the poses of s^{k+1} (in)
    double *gs0;            // [S][NS] accumulated adjoint of the initial states
    void *scratch;
    const long long *scratch0;
};

template <typename T>
struct AdjPairArgs {
    const ScenMeta *meta;
    const Tile *tiles;
    Geom<T> g;
    const T *pose;          // [PK][Qtot] poses of s^k
    int Qtot;
    long long P;
    T prox;
    const int *iters;
    int k;
    const T *y_k, *y_k1;    // y^k (proximal centre, head), y^{k+1} (QP solution)
    const T *zx_k;          // zeta^k, xi^k
    const T *ybar_in;       // [NY][P] adjoint of y^{k+1} from iteration k+1
    T *ybar_out;            // [NY][P] adjoint of y^k (partial: proximal centre and head)
    T *zb, *xb;             // [P], [D][P] running adjoints of zeta and xi
    const T *statsb;        // [NSTAT][Qtot]
    T *poseb;               // [PK][Qtot] adjoint of the poses of s^k (out)
    double *gd;             // [M_tot][FO] accumulated adjoint of the obstacle offsets
};

template <typename T>
struct AdjAlphaArgs {
    const ScenMeta *meta;
    const Tile *tiles;
    Geom<T> g;
    const T *pose;          // [PK][Qtot] poses of the returned states
    int Qtot;
    long long P;
    const T *grad_alpha;    // [P]
    T *poseb;               // [PK][Qtot] out: adjoint of those poses
    double *gd;             // [M_tot][FO] accumulated adjoint of the obstacle offsets
};

// closed-loop receding-horizon control (oca_mpc_run)
template <typename T>
struct MpcArgs {
    const ScenMeta *meta;
    Geom<T> g;
    DevModel<T> model;
    const T *ref;          // [S][T_ref][NS] reference of every control step
    int T_ref;
    const T *obs_center;   // [M_tot][D]
    T win[3];              // sensing half-widths per axis (<= 0: no limit on that axis)
    T *x;                  // [S][NS] true state
    T *s, *u, *s_ref;      // the scene's state arrays (warm start, window)
    T *y, *zeta, *xi;      // pair arrays
    long long P;
    int FR, FO;
    unsigned char *mask;   // [M_tot] sensed obstacles of this step
    T *x_hist, *u_hist;    // [S][n_steps + 1][NS], [S][n_steps][NU]
    int n_steps;
    int *collided;         // [S] first control step whose true state collides, or -1
    int *iters_hist;       // [S][n_steps]
    const int *iters;      // [S] iterations of this step's solve
    int c;                 // control step
};

// the paper's Lemke route for the pair QPs (comparison kernel)
template <typename T>
struct LemkeArgs {
    const ScenMeta *meta;
    Geom<T> g;
    const T *pose;       // [PK][Qtot]
    int Qtot;
    long long P;
    int n_scen;
    const T *zeta, *xi, *y_in;
    T *y_out, *v_out, *obj_out;
    int *status_out;
    T prox;
};

}  // namespace oca
