// Scale-based collision detection of one scenario without any allocation.
//
// oca_scale_detect_batch needs an oca_scene, whose creation allocates device
// memory (metadata, work tiles, the pose buffer).  Some callers cannot
// allocate at all: a real-time control loop that must not enter the CUDA
// allocator (it can block or synchronise the device), or a plugin whose host
// forbids heap use.
// oca_scale_detect_noalloc serves them: its scratch (the face counts and part
// links copied from the host metadata, and the poses of the scenario's
// (part, t) lanes) lives in the file-scope device array below, the scenario's
// sizes travel by value as kernel arguments and the work tiles are implicit
// (tile k covers lanes 32k .. 32k + 31).
#include <cstring>

#include "oca_common.cuh"
#include "oca_models.cuh"
#include "oca_solvers.cuh"

namespace {

using namespace oca;

// Scratch shared by every call on a device: 1 MiB holding the face counts and
// part links (copied from the host metadata) and the poses of the
// parts x N lanes, (dim + dim^2) values each.
constexpr size_t kNoallocScratchBytes = size_t(1) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

struct OneScen {
    int N, M, NP, Q;
};

template <typename T, int KIND>
__global__ void k_pose_one(OneScen sc, Geom<T> g, DevModel<T> model, const T *states, T *pose) {
    constexpr int D = MDims<KIND>::D, NS = MDims<KIND>::NS;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= sc.Q) return;
    const int part = q / sc.N, t = q % sc.N + 1;
    T st[NS], off[D], rho[D], R[D * D];
#pragma unroll
    for (int i = 0; i < NS; ++i) st[i] = states[(long long)t * NS + i];
#pragma unroll
    for (int i = 0; i < D; ++i) off[i] = g.part_off[part * D + i];
    part_pose<T, KIND>(model, g.part_link[part], off, st, rho, R, nullptr, nullptr, nullptr);
#pragma unroll
    for (int i = 0; i < D; ++i) pose[(long long)i * sc.Q + q] = rho[i];
#pragma unroll
    for (int i = 0; i < D * D; ++i) pose[(long long)(D + i) * sc.Q + q] = R[i];
}

template <typename T, int D>
__global__ void k_scale_one(OneScen sc, Geom<T> g, const T *pose, T *alpha, T *lambda, T *mu, int *verdict,
                            int *status) {
    constexpr int V = D + 1;
    const int lane = threadIdx.x, warp = threadIdx.y, W = blockDim.y;
    const int q = blockIdx.x * 32 + lane;
    if (q >= sc.Q) return;
    const long long P = (long long)sc.M * sc.Q;
    Lane<T, D> L;
#pragma unroll
    for (int i = 0; i < D; ++i) L.rho[i] = pose[(long long)i * sc.Q + q];
#pragma unroll
    for (int i = 0; i < D * D; ++i) L.R[i] = pose[(long long)(D + i) * sc.Q + q];
    const int part = q / sc.N;
    L.A = g.part_A + (long long)part * g.FR * D;
    L.b = g.part_b + (long long)part * g.FR;
    L.nr = g.part_nf[part];
    for (int j = warp; j < sc.M; j += W) {
        L.C = g.obs_C + (long long)j * g.FO * D;
        L.d = g.obs_d + (long long)j * g.FO;
        L.no = g.obs_nf[j];
        const long long p = (long long)j * sc.Q + q;
        int bas[V];
        T xB[V], a;
        int st = lp_solve<T, D>(L, bas, xB, a);
        if (!(a == a)) st = OCA_PAIR_NONFINITE;
        alpha[p] = a;
        if (verdict) verdict[p] = a >= T(1) ? 1 : 0;
        if (status) status[p] = st;
        if (lambda)
            for (int k = 0; k < L.nr; ++k) {
                T v = T(0);
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (bas[i] == k) v = xB[i];
                lambda[(long long)k * P + p] = v;
            }
        if (mu)
            for (int m = 0; m < L.no; ++m) {
                T v = T(0);
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (bas[i] == L.nr + m) v = xB[i];
                mu[(long long)m * P + p] = v;
            }
    }
}

template <typename T>
oca_status run(const oca_scene_desc *d, const oca_model *m, void *scratch, const void *states, void *alpha,
               void *lambda, void *mu, int32_t *verdict, int32_t *status, cudaStream_t st) {
    OneScen sc;
    sc.N = d->horizon[0];
    sc.M = d->obs_begin[1];
    sc.NP = d->part_begin[1];
    sc.Q = sc.NP * sc.N;
    Geom<T> g;
    g.obs_C = static_cast<const T *>(d->obs_C);
    g.obs_d = static_cast<const T *>(d->obs_d);
    g.part_A = static_cast<const T *>(d->part_A);
    g.part_b = static_cast<const T *>(d->part_b);
    g.part_off = static_cast<const T *>(d->part_off);
    g.FO = d->fo_max;
    g.FR = d->fr_max;
    // face counts and part links: host metadata, copied into the head of the scratch
    int *ints = static_cast<int *>(scratch);
    const size_t nint = (size_t)sc.M + 2 * (size_t)sc.NP;
    if (cudaMemcpyAsync(ints, d->obs_nf, sizeof(int) * sc.M, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ints + sc.M, d->part_nf, sizeof(int) * sc.NP, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ints + sc.M + sc.NP, d->part_link, sizeof(int) * sc.NP, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return OCA_ERR_CUDA;
    g.obs_nf = ints;
    g.part_nf = ints + sc.M;
    g.part_link = ints + sc.M + sc.NP;
    scratch = static_cast<unsigned char *>(scratch) + ((nint * sizeof(int) + 255) / 256) * 256;
    DevModel<T> dm;
    std::memset(&dm, 0, sizeof(dm));
    dm.kind = m->kind;
    dm.dt = T(m->dt);
    for (int i = 0; i < 8; ++i) dm.p[i] = T(m->param[i]);
    T *pose = static_cast<T *>(scratch);
    const unsigned blocks = (unsigned)((sc.Q + 127) / 128);
    switch (m->kind) {
        case 0: k_pose_one<T, 0><<<blocks, 128, 0, st>>>(sc, g, dm, static_cast<const T *>(states), pose); break;
        case 1: k_pose_one<T, 1><<<blocks, 128, 0, st>>>(sc, g, dm, static_cast<const T *>(states), pose); break;
        default: k_pose_one<T, 2><<<blocks, 128, 0, st>>>(sc, g, dm, static_cast<const T *>(states), pose); break;
    }
    if (cudaGetLastError() != cudaSuccess) return OCA_ERR_CUDA;
    const int W = sc.M >= 32 ? 4 : (sc.M >= 8 ? 2 : 1);
    const unsigned tiles = (unsigned)((sc.Q + 31) / 32);
    if (d->dim == 2)
        k_scale_one<T, 2><<<tiles, dim3(32, W), 0, st>>>(sc, g, pose, static_cast<T *>(alpha), static_cast<T *>(lambda),
                                                        static_cast<T *>(mu), verdict, status);
    else
        k_scale_one<T, 3><<<tiles, dim3(32, W), 0, st>>>(sc, g, pose, static_cast<T *>(alpha), static_cast<T *>(lambda),
                                                        static_cast<T *>(mu), verdict, status);
    return cudaGetLastError() == cudaSuccess ? OCA_OK : OCA_ERR_CUDA;
}

}  // namespace

extern "C" oca_status oca_scale_detect_noalloc(const oca_scene_desc *desc, const oca_model *model,
                                               const void *states, void *alpha, void *lambda, void *mu,
                                               int32_t *verdict, int32_t *status, void *stream) {
    if (!desc || !model || !states || !alpha) return OCA_ERR_INVALID_ARGUMENT;
    if (desc->n_scen != 1 || (desc->dim != 2 && desc->dim != 3)) return OCA_ERR_INVALID_ARGUMENT;
    if (desc->dtype != OCA_F32 && desc->dtype != OCA_F64) return OCA_ERR_INVALID_ARGUMENT;
    if (!desc->obs_begin || !desc->part_begin || !desc->horizon || !desc->obs_nf || !desc->part_nf ||
        !desc->part_link || !desc->obs_C || !desc->obs_d || !desc->part_A || !desc->part_b || !desc->part_off)
        return OCA_ERR_INVALID_ARGUMENT;
    if (model->kind < 0 || model->kind > 2 || (model->kind == 2) != (desc->dim == 3)) return OCA_ERR_INVALID_ARGUMENT;
    if (desc->fo_max < 1 || desc->fr_max < 1) return OCA_ERR_INVALID_ARGUMENT;
    if (desc->fo_max > OCA_MAX_OBS_FACES || desc->fr_max > OCA_MAX_PART_FACES) return OCA_ERR_CAPACITY;
    const int N = desc->horizon[0], M = desc->obs_begin[1], NP = desc->part_begin[1];
    if (N < 1 || M < 1 || NP < 1 || desc->obs_begin[0] != 0 || desc->part_begin[0] != 0)
        return OCA_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < M; ++i)
        if (desc->obs_nf[i] < 1 || desc->obs_nf[i] > desc->fo_max) return OCA_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < NP; ++i) {
        if (desc->part_nf[i] < desc->dim + 1 || desc->part_nf[i] > desc->fr_max) return OCA_ERR_INVALID_ARGUMENT;
        if (desc->part_link[i] < 0 || desc->part_link[i] > 1 || (desc->dim == 3 && desc->part_link[i] != 0))
            return OCA_ERR_INVALID_ARGUMENT;
    }
    const size_t es = desc->dtype == OCA_F64 ? sizeof(double) : sizeof(float);
    const size_t ints = (((size_t)M + 2 * (size_t)NP) * sizeof(int) + 255) / 256 * 256;
    const size_t need = ints + (size_t)(desc->dim + desc->dim * desc->dim) * (size_t)NP * (size_t)N * es;
    if (need > kNoallocScratchBytes) return OCA_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OCA_ERR_CUDA;
    if (!g_scratch_ptr[dev]) {
        // once per device, with that device current: the host-side name of the
        // array is not a device address, so look the address up
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return OCA_ERR_CUDA;
        g_scratch_ptr[dev] = ptr;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (desc->dtype == OCA_F32)
        return run<float>(desc, model, g_scratch_ptr[dev], states, alpha, lambda, mu, verdict, status, st);
    return run<double>(desc, model, g_scratch_ptr[dev], states, alpha, lambda, mu, verdict, status, st);
}
