// C ABI of the FEWHA reconstructor (declared in include/fewha.h): instance set-up,
// the per-frame sequence of Algorithm 1 (optionally replayed as a CUDA graph) and
// the operator entry points used by the tests and the autograd layer.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <initializer_list>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "fewha_batch.h"
#ifdef FEWHA_NVTX
#include <nvtx3/nvToolsExt.h>
#endif
#include "fewha_lsfit.cuh"
#include "fewha_persist.cuh"

using namespace fewha;

// Optional NVTX ranges around the entry points (build with -DFEWHA_NVTX), so that a
// timeline tool shows each call's span over its kernels; compiled out otherwise.
#ifdef FEWHA_NVTX
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
#define FEWHA_RANGE(name) NvtxRange fewha_nvtx_range_(name)
#else
#define FEWHA_RANGE(name) ((void)0)
#endif

namespace {

thread_local std::string g_create_error;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

constexpr int NPART_MAX = 512;
constexpr int PQ_SCRATCH_SLOT = FEWHA_MAX_ITERS;   // p.q slot of the explicit r0 apply
static_assert(AUG_MAX == FEWHA_AUG_MAX_ITERS, "augmented PCG direction count");

}  // namespace

// Least-squares fit over fitting directions (fewha_fit_ls): the configuration whose tables
// are on the device, those tables (see LsfitHost) and the CG vectors.  Buffers grow with the
// configuration and are owned by the handle's allocation list.
struct LsfitDev {
    std::vector<double> key;
    LsfitHost host;
    unsigned char* mask = nullptr;
    int *ly0 = nullptr, *lx0 = nullptr, *my0 = nullptr, *mx0 = nullptr;
    int *ylo = nullptr, *yhi = nullptr, *xlo = nullptr, *xhi = nullptr;
    void *lfy = nullptr, *lfx = nullptr, *mfy = nullptr, *mfx = nullptr;
    void *v = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
    double* part = nullptr;
    double* msum = nullptr;
    double* sc = nullptr;
    int* state = nullptr;
    size_t cap_pix = 0, cap_l = 0, cap_lf = 0, cap_m = 0, cap_mf = 0, cap_rng = 0, cap_v = 0;
};

struct fewha_handle {
    int device = 0;
    int precision = 32;
    size_t esz = 4;
    fewha_params params{};
    HostSetup setup;
    std::vector<double> weights;   // current layer Cn2 weights
    std::vector<void*> allocs;
    std::vector<size_t> alloc_sizes;   // bytes of each of allocs
    // device tables (precision independent)
    int *pi0y = nullptr, *pi0x = nullptr, *ry_lo = nullptr, *ry_hi = nullptr, *rx_lo = nullptr,
        *rx_hi = nullptr, *sidx = nullptr, *cidx = nullptr, *di0 = nullptr, *dr_lo = nullptr,
        *dr_hi = nullptr, *basis_off = nullptr;
    double *pfy64 = nullptr, *pfx64 = nullptr, *basis = nullptr, *D64 = nullptr, *Jdata = nullptr,
           *J64 = nullptr, *rzpart = nullptr, *pqpart = nullptr, *rztot = nullptr, *pqtot = nullptr;
    unsigned* status = nullptr;
    unsigned* count = nullptr;
    int npart = 1;
    // typed device arrays (float or double per precision)
    void *pfy = nullptr, *pfx = nullptr, *dfw = nullptr, *D = nullptr, *Jinv = nullptr;
    void *c = nullptr, *b = nullptr, *b_prev = nullptr, *r = nullptr, *z = nullptr, *p = nullptr,
         *q = nullptr, *phi = nullptr, *phic = nullptr, *u = nullptr, *a_prev = nullptr, *dm_tmp = nullptr,
         *s_tmp = nullptr, *c_tmp = nullptr, *cgrad = nullptr, *lam = nullptr;
    double* gdot = nullptr;           // per-layer sums of the backward pass
    // closed loop (FEWHA_FLAG_CLOSED_LOOP): DM projection tables, pseudo-open-loop slopes
    // and the commands of the frame before (a^(i-1))
    int *qi0y = nullptr, *qi0x = nullptr;
    void *qfy = nullptr, *qfx = nullptr, *s_pol = nullptr, *a_old = nullptr, *dm_nodes = nullptr;
    bool grad_ready = false;          // a converged reconstruction is held in cgrad
    bool have_cgrad = false;          // cgrad / lam hold earlier solutions (warm starts)
    bool have_lam = false;
    double grad_tol = 0.0;
    int grad_max_iters = 0;
    bool have_prev = false;
    // augmented PCG (FEWHA_FLAG_AUGMENTED): two sets of AUG_MAX directions and images
    // (stride aug_ld), a frame writes set aug_set and reads the other (aug_m directions)
    void *Pd[2] = {nullptr, nullptr}, *Qd[2] = {nullptr, nullptr};
    double* pqd[2] = {nullptr, nullptr};
    double *augpart = nullptr, *augtot = nullptr;
    size_t aug_ld = 0;
    int aug_set = 0, aug_m = 0;
    // frame-graph cache
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[2] = {};    // plain frames: [explicit r0, warm r0]
    cudaGraphExec_t gaug[4] = {};     // augmented frames: [2 * set + (directions present)]
    int warm_run = 0;                 // frames in a row on the warm-residual recurrence
    // reverse pass through the fixed-iteration frame: its recorded vectors (allocated on use)
    void* vjp = nullptr;
    size_t vjp_cap = 0;
    const void* g_s = nullptr;
    void* g_x = nullptr;
    void* g_dm = nullptr;
    bool g_warm = false;
    std::string err;
    size_t smem_layer = 0, smem_sensor = 0;
    // cluster kernels of the hot path
    ClLayout lay_fwd{}, lay_inv{};
    SensorLayout lay_sen{};
    size_t smem_fwd = 0, smem_inv = 0, smem_sen = 0, smem_proj = 0, smem_projT = 0;
    int kmax = KMAX;                  // most aperture rows / columns touching one layer row / column
    // (sensor, layer) pair terms of P and P^T
    int* box = nullptr;
    int* ytab = nullptr;              // band-run table of the forward kernel (PairBufs::ytab)
    void* ptw = nullptr;              // adjoint-projection weights (PairBufs::tw), T
    void* tailop = nullptr;           // the 8 x 8 tail levels as one matrix (Desc::tailop), T
    int* pti = nullptr;               // their first index and count (PairBufs::ti)
    std::vector<int> box_host;
    void* pairV = nullptr;
    void* pairY = nullptr;
    int pvs = 0, pvslot = 0, pyslot = 0;
    // batches this instance belongs to, and a counter of parameter updates (a batch
    // rebuilds its copy of the descriptor when it changes)
    std::vector<fewha_batch*> batches;
    unsigned version = 0;
    // creation inputs, and the double-precision twin of a single-precision handle that
    // forms the true residuals of its converged solves (created on first use)
    fewha_telescope tel_in{};
    std::vector<fewha_wfs> wfs_in;
    std::vector<fewha_layer> layers_in;
    std::vector<fewha_dm> dms_in;
    fewha_handle* twin = nullptr;
    // persistent frame (FEWHA_FLAG_PERSISTENT): grid-barrier words (arrivals, abort), the
    // clusters of its launch (0 = not set up yet), its dynamic shared memory, wait limits
    unsigned* gbar = nullptr;
    int pers_ncl = 0;
    size_t smem_frame = 0;
    unsigned wait_limit = 1u << 20;
    unsigned wait_extra = 0;
    LsfitDev* lsf = nullptr;
};

struct fewha_batch {
    std::vector<fewha_handle*> h;   // members (an entry is cleared when its handle is destroyed)
    std::vector<unsigned> ver;      // member versions the plan was built with
    int precision = 32;
    int device = 0;
    bool dead = false;
    bool registry = false;          // owned by the fewha_reconstruct_batched cache
    std::string err;
    fewha_batch_config cfg{0, 1, 1, 0, 0, 0};
    // current plan: one device block [instances | work lists | argument table] and a graph
    bool have_plan = false;
    bool plan_warm = false;
    fewha_batch_config plan_cfg{0, 0, 0, 0, 0, 0};
    void* dev = nullptr;
    size_t args_off = 0;
    std::vector<unsigned char> args_host;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t branch[FEWHA_BATCH_MAX_GROUPS] = {};
    cudaEvent_t ev[FEWHA_BATCH_MAX_GROUPS] = {};
};

namespace {

int fail(fewha_handle* H, int code, const std::string& msg) {
    if (H) H->err = msg;
    return code;
}

int cuda_fail(fewha_handle* H, cudaError_t e, const char* where) {
    return fail(H, FEWHA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(H, e_, where); \
    } while (0)

// Allocation-failure injection (fewha_test_fail_alloc): the number of device allocations
// of this thread still to succeed before one fails; -1 = off.
thread_local int g_fail_countdown = -1;

// Every device allocation of the library goes through here.
cudaError_t dev_malloc(void** p, size_t bytes) {
    if (g_fail_countdown >= 0) {
        if (g_fail_countdown == 0) {
            g_fail_countdown = -1;
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        --g_fail_countdown;
    }
    return cudaMalloc(p, bytes);
}

void track(fewha_handle* H, void* p, size_t bytes) {
    H->allocs.push_back(p);
    H->alloc_sizes.push_back(bytes);
}

template <class X>
int dalloc(fewha_handle* H, X** ptr, size_t count) {
    void* p = nullptr;
    const size_t bytes = count * sizeof(X) > 0 ? count * sizeof(X) : 16;
    if (dev_malloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(H, FEWHA_ERR_OOM, "device allocation failed");
    }
    cudaMemset(p, 0, bytes);
    track(H, p, bytes);
    *ptr = static_cast<X*>(p);
    return FEWHA_OK;
}

int talloc(fewha_handle* H, void** ptr, size_t count) {
    void* p = nullptr;
    // 16 spare elements: the 16-byte staging copies may read up to one chunk past a vector
    const size_t bytes = (count + 16) * H->esz;
    if (dev_malloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(H, FEWHA_ERR_OOM, "device allocation failed");
    }
    cudaMemset(p, 0, bytes);
    track(H, p, bytes);
    *ptr = p;
    return FEWHA_OK;
}

template <class X>
int upload(fewha_handle* H, X* dst, const std::vector<X>& src) {
    if (src.empty()) return FEWHA_OK;
    CK(cudaMemcpy(dst, src.data(), src.size() * sizeof(X), cudaMemcpyHostToDevice), "upload");
    return FEWHA_OK;
}

template <class T>
Desc<T> make_desc(const fewha_handle* H) {
    const HostSetup& s = H->setup;
    Desc<T> d;
    std::memset(&d, 0, sizeof(d));
    d.n_layers = static_cast<int>(s.L.size());
    d.n_wfs = static_cast<int>(s.G.size());
    d.n_dms = static_cast<int>(s.Mi.size());
    d.n_c = s.n_c;
    d.n_s = s.n_s;
    d.n_nodes = s.n_nodes;
    d.n_act = s.n_act;
    d.max_n = s.max_n;
    d.max_N = s.max_N;
    for (int l = 0; l < d.n_layers; ++l) d.L[l] = s.L[l];
    for (int g = 0; g < d.n_wfs; ++g) d.G[g] = s.G[g];
    for (int m = 0; m < d.n_dms; ++m) {
        d.Mi[m] = s.Mi[m];
        for (int l = 0; l < d.n_layers; ++l) d.fitw[m][l] = T(s.fitw[m][l]);
    }
    d.alpha = T(H->params.alpha);
    d.gain = T(H->params.gain);
    d.pi0y = H->pi0y;
    d.pi0x = H->pi0x;
    d.pfy = static_cast<const T*>(H->pfy);
    d.pfx = static_cast<const T*>(H->pfx);
    d.ry_lo = H->ry_lo;
    d.ry_hi = H->ry_hi;
    d.rx_lo = H->rx_lo;
    d.rx_hi = H->rx_hi;
    d.sidx = H->sidx;
    d.cidx = H->cidx;
    d.di0 = H->di0;
    d.dfw = static_cast<const T*>(H->dfw);
    d.dr_lo = H->dr_lo;
    d.dr_hi = H->dr_hi;
    d.D = static_cast<const T*>(H->D);
    d.Jinv = static_cast<const T*>(H->Jinv);
    for (int l = 0; l < d.n_layers && !s.dlev.empty(); ++l)
        for (int k = 0; k <= MAXLEV; ++k) d.Dlev[l][k] = T(s.dlev[l * (MAXLEV + 1) + k]);
    d.tailop = static_cast<const T*>(H->tailop);
    for (int g = 0; g < d.n_wfs; ++g)
        for (int l = 0; l < d.n_layers; ++l)
            for (int k = 0; k < 4; ++k) d.box[g][l][k] = H->box_host[(g * MAXL + l) * 4 + k];
    return d;
}

// Launch of a hot-path kernel, with programmatic stream serialization if the handle asks
// for it (FEWHA_FLAG_PDL; the kernels then wait for their predecessor on the device).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(const fewha_handle* H, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = (H->params.flags & FEWHA_FLAG_PDL) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------- step recording
// A batched frame runs the single-instance frame sequence of every instance: while a
// recorder is set on this thread, the launchers below append their step (kind and
// arguments) to it instead of launching.
template <class T>
struct BStep {
    int kind;
    ClArgs<T> cl;
    SensorArgs<T> sa;
    VecArgs<T> va;
    const T* ptr;
    FitArgs<T> fa;
};

template <class T>
struct Recorder {
    std::vector<BStep<T>> steps;
};

thread_local void* g_recorder = nullptr;

template <class T>
Recorder<T>* recorder() {
    return static_cast<Recorder<T>*>(g_recorder);
}

template <class T>
BStep<T>& record(int kind) {
    BStep<T> st;
    std::memset(&st, 0, sizeof(st));
    st.kind = kind;
    recorder<T>()->steps.push_back(st);
    return recorder<T>()->steps.back();
}

// ---------------------------------------------------------------- launchers
template <class T, int SRC, int DST, bool PUPD>
int launch_layer(fewha_handle* H, const Desc<T>& d, const LayerArgs<T>& a, cudaStream_t st) {
    k_layer<T, SRC, DST, PUPD><<<d.n_layers, BLK, H->smem_layer, st>>>(d, a);
    CK(cudaGetLastError(), "k_layer launch");
    return FEWHA_OK;
}

template <class T, int SRC, bool WEIGHT, int DST>
int launch_sensor(fewha_handle* H, const Desc<T>& d, const T* in, T* out, cudaStream_t st) {
    SensorArgs<T> a{in, out, H->status};
    k_sensor<T, SRC, WEIGHT, DST><<<d.n_wfs, BLK, H->smem_sensor, st>>>(d, a);
    CK(cudaGetLastError(), "k_sensor launch");
    return FEWHA_OK;
}

PcgSlots pcg_slots(fewha_handle* H) {
    PcgSlots p;
    p.rzpart = H->rzpart;
    p.pqpart = H->pqpart;
    p.rztot = H->rztot;
    p.pqtot = H->pqtot;
    p.count = H->count;
    p.npart = H->npart;
    return p;
}

template <class T>
VecArgs<T> vec_args(fewha_handle* H, T* c, int iter) {
    VecArgs<T> v;
    v.c = c;
    v.r = static_cast<T*>(H->r);
    v.z = static_cast<T*>(H->z);
    v.p = static_cast<T*>(H->p);
    v.q = static_cast<const T*>(H->q);
    v.b = static_cast<const T*>(H->b);
    v.b_prev = static_cast<T*>(H->b_prev);
    v.Jinv = static_cast<const T*>(H->Jinv);
    v.pcg = pcg_slots(H);
    v.iter = iter;
    v.pq_cnt = 0;
    v.defer_rz = 0;
    v.phic = nullptr;
    v.phip = nullptr;
    return v;
}

template <class T>
LayerArgs<T> layer_args(fewha_handle* H, const T* in, T* out) {
    LayerArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.in = in;
    a.out = out;
    a.pcg = pcg_slots(H);
    return a;
}

template <class T>
ClArgs<T> cl_args(fewha_handle* H, const T* in, T* out) {
    ClArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.in = in;
    a.out = out;
    a.pcg = pcg_slots(H);
    return a;
}

template <class T>
PairBufs<T> pair_bufs(fewha_handle* H) {
    PairBufs<T> pb;
    pb.V = static_cast<T*>(H->pairV);
    pb.Y = static_cast<T*>(H->pairY);
    pb.vs = H->pvs;
    pb.vslot = H->pvslot;
    pb.yslot = H->pyslot;
    pb.box = H->box;
    pb.ytab = reinterpret_cast<const int4*>(H->ytab);
    pb.tw = static_cast<const T*>(H->ptw);
    pb.ti = reinterpret_cast<const int2*>(H->pti);
    return pb;
}

template <class T>
int launch_proj(fewha_handle* H, const Desc<T>& d, const T* phi, cudaStream_t st) {
    if (recorder<T>()) {
        record<T>(BK_PROJ).ptr = phi;
        return FEWHA_OK;
    }
    CK(launch_k(H, k_proj<T>, dim3(d.n_wfs, d.n_layers), dim3(cblk<T>()), H->smem_proj, st, d, phi,
                pair_bufs<T>(H)),
       "k_proj launch");
    return FEWHA_OK;
}

template <class T>
int launch_projT(fewha_handle* H, const Desc<T>& d, const T* u, cudaStream_t st) {
    if (recorder<T>()) {
        record<T>(BK_PROJT).ptr = u;
        return FEWHA_OK;
    }
    if (H->kmax <= 4)
        CK(launch_k(H, k_projT<T, 4>, dim3(d.n_wfs, d.n_layers), dim3(cblk<T>()), H->smem_projT, st, d, u,
                    pair_bufs<T>(H)),
           "k_projT launch");
    else
        CK(launch_k(H, k_projT<T, KMAX>, dim3(d.n_wfs, d.n_layers), dim3(cblk<T>()), H->smem_projT, st, d, u,
                    pair_bufs<T>(H)),
           "k_projT launch");
    return FEWHA_OK;
}

template <class T, int SRC, int DST>
int launch_fwd(fewha_handle* H, const Desc<T>& d, const ClArgs<T>& a, cudaStream_t st) {
    if (recorder<T>()) {
        if (SRC != LSRC_NODES || (DST != LDST_APPLY && DST != LDST_COEF && DST != LDST_RESID_INIT))
            return fail(H, FEWHA_ERR_INVALID_ARG, "step without a batched form");
        record<T>(DST == LDST_APPLY ? BK_FWD_APPLY : DST == LDST_RESID_INIT ? BK_FWD_RINIT : BK_FWD_COEF).cl = a;
        return FEWHA_OK;
    }
    CK(launch_k(H, k_cl_fwd<T, SRC, DST>, dim3(CL, d.n_layers), dim3(cblk<T>()), H->smem_fwd, st, d, a,
                H->lay_fwd, pair_bufs<T>(H)),
       "k_cl_fwd launch");
    return FEWHA_OK;
}

template <class T, int PUPD>
int launch_inv(fewha_handle* H, const Desc<T>& d, const ClArgs<T>& a, cudaStream_t st) {
    if (recorder<T>()) {
        record<T>(PUPD ? BK_INV_UPD : BK_INV).cl = a;
        return FEWHA_OK;
    }
    CK(launch_k(H, k_cl_inv<T, PUPD>, dim3(CL, d.n_layers), dim3(cblk<T>()), H->smem_inv, st, d, a,
                H->lay_inv),
       "k_cl_inv launch");
    return FEWHA_OK;
}

template <class T, int SRC>
int launch_csensor(fewha_handle* H, const Desc<T>& d, const T* in, T* out, cudaStream_t st) {
    SensorArgs<T> a{in, out, H->status};
    if (recorder<T>()) {
        record<T>(SRC == SSRC_PHI ? BK_SEN_PHI : SRC == SSRC_RESID ? BK_SEN_RESID : BK_SEN_SLOPES).sa = a;
        return FEWHA_OK;
    }
    CK(launch_k(H, k_cl_sensor<T, SRC>, dim3(CL, d.n_wfs), dim3(cblk<T>()), H->smem_sen, st, d, a,
                H->lay_sen, pair_bufs<T>(H)),
       "k_cl_sensor launch");
    return FEWHA_OK;
}

// Deferred dot totals of one apply inside the frame's PCG (see ClArgs): the forward
// kernel's p.q total is left to the CG update, and the inverse kernel forms the r.z total
// of slot rz_slot from rz_cnt shares at rz_parts (rz_cnt = 0: none).
struct Defer {
    bool pq = false;
    const double* rz_parts = nullptr;
    int rz_cnt = 0;
    int rz_slot = 0;
};

// q = M x (Eq. 6); the p.q partials go to slot `slot` (PQ_SLOTS doubles per slot).
// With pupdate, x is the CG direction p, first advanced to z + beta p (iteration `slot`).
template <class T>
int enqueue_apply(fewha_handle* H, const Desc<T>& d, const T* x, T* qout, int slot, bool pupdate,
                  cudaStream_t st, const Defer& df = Defer()) {
    T* phi = static_cast<T*>(H->phi);
    T* u = static_cast<T*>(H->u);
    int rc;
    ClArgs<T> a = cl_args<T>(H, x, phi);
    a.zero_piston = 1;                 // the data path's input leaves the piston out
    a.rz_parts = df.rz_parts;
    a.rz_cnt = df.rz_cnt;
    a.rz_slot = df.rz_slot;
    if (pupdate) {
        a.pupd = static_cast<T*>(H->p);
        a.zupd = static_cast<const T*>(H->z);
        a.iter = slot;
        rc = launch_inv<T, 1>(H, d, a, st);
    } else {
        rc = launch_inv<T, 0>(H, d, a, st);
    }
    if (rc) return rc;
    if ((rc = launch_proj<T>(H, d, phi, st))) return rc;
    if ((rc = launch_csensor<T, SSRC_PHI>(H, d, phi, u, st))) return rc;
    if ((rc = launch_projT<T>(H, d, u, st))) return rc;
    ClArgs<T> b = cl_args<T>(H, u, qout);
    b.pin = x;
    b.iter = slot;
    b.zero_piston = 1;
    b.defer_total = df.pq ? 1 : 0;
    return launch_fwd<T, LSRC_NODES, LDST_APPLY>(H, d, b, st);
}

// q = M p_new with the direction update of the augmented PCG (Sec. 3.4) fused into the
// inverse kernel: p_new = z + beta p_old - sum_j mu_j P_j (beta from rz slots `slot` and
// `slot - 1`; no p_old, and beta = 0, when pold is null; the m directions of `aug`).
template <class T>
int enqueue_apply_aug(fewha_handle* H, const Desc<T>& d, const T* pold, T* pnew, const T* z, T* qout, int slot,
                      const AugArgs<T>& aug, cudaStream_t st, const Defer& df = Defer(),
                      int aug_pcnt = 0) {
    T* phi = static_cast<T*>(H->phi);
    T* u = static_cast<T*>(H->u);
    int rc;
    ClArgs<T> a = cl_args<T>(H, nullptr, phi);
    a.zero_piston = 1;
    a.pupd = const_cast<T*>(pold);       // read only by the augmented update
    a.zupd = z;
    a.pout = pnew;
    a.iter = slot;
    a.augP = aug.P;
    a.aug_tot = aug.tot;
    a.aug_pq = aug.pq;
    a.aug_ld = aug.ld;
    a.aug_m = aug.m;
    a.aug_parts = aug.part;
    a.aug_pcnt = aug_pcnt;
    a.rz_parts = df.rz_parts;
    a.rz_cnt = df.rz_cnt;
    a.rz_slot = df.rz_slot;
    if ((rc = launch_inv<T, 2>(H, d, a, st))) return rc;
    if ((rc = launch_proj<T>(H, d, phi, st))) return rc;
    if ((rc = launch_csensor<T, SSRC_PHI>(H, d, phi, u, st))) return rc;
    if ((rc = launch_projT<T>(H, d, u, st))) return rc;
    ClArgs<T> b = cl_args<T>(H, u, qout);
    b.pin = pnew;
    b.iter = slot;
    b.zero_piston = 1;
    b.defer_total = df.pq ? 1 : 0;
    return launch_fwd<T, LSRC_NODES, LDST_APPLY>(H, d, b, st);
}

// r = b - M c0 (as enqueue_apply, then V_INIT) with the initial residual's vector step fused
// into the forward kernel's epilogue: r0, z0 = J^-1 r0, p0 = z0, b_prev = b, r.z into slot 0
// (with `defer`, only its n_layers * CL shares, at the start of the r.z slots).
template <class T>
int enqueue_apply_init(fewha_handle* H, const Desc<T>& d, T* c, cudaStream_t st, bool defer = false) {
    const T* x = c;
    const int slot = PQ_SCRATCH_SLOT;
    const bool pupdate = false;
    T* phi = static_cast<T*>(H->phi);
    T* u = static_cast<T*>(H->u);
    int rc;
    ClArgs<T> a = cl_args<T>(H, x, phi);
    a.zero_piston = 1;
    if (pupdate) {
        a.pupd = static_cast<T*>(H->p);
        a.zupd = static_cast<const T*>(H->z);
        a.iter = slot;
        rc = launch_inv<T, 1>(H, d, a, st);
    } else {
        rc = launch_inv<T, 0>(H, d, a, st);
    }
    if (rc) return rc;
    if ((rc = launch_proj<T>(H, d, phi, st))) return rc;
    if ((rc = launch_csensor<T, SSRC_PHI>(H, d, phi, u, st))) return rc;
    if ((rc = launch_projT<T>(H, d, u, st))) return rc;
    ClArgs<T> b = cl_args<T>(H, u, static_cast<T*>(H->q));
    b.pin = x;
    b.iter = slot;
    b.zero_piston = 1;
    b.vr = static_cast<T*>(H->r);
    b.vz = static_cast<T*>(H->z);
    b.vp = static_cast<T*>(H->p);
    b.vb = static_cast<const T*>(H->b);
    b.vbprev = static_cast<T*>(H->b_prev);
    b.vj = static_cast<const T*>(H->Jinv);
    b.rzslot = 0;
    b.rzp = H->rzpart;
    b.defer_total = defer ? 1 : 0;
    return launch_fwd<T, LSRC_NODES, LDST_APPLY_INIT>(H, d, b, st);
}

// r0 = b - M c0 formed in one chain, from the slopes' residual: the sensor kernel takes
// C^-1 (s - Gamma P phi0) (phi0 = W^T c0, its piston left out), the adjoint projection and
// the forward kernel give r0 = W P^T Gamma^T C^-1 (s - Gamma P phi0) - alpha D c0 and the
// initial residual's vector step (z0, p0, r.z in slot 0, only shares with `defer`).  By
// linearity this is b - M c0 of Algorithm 1 without forming b: 5 kernels instead of the
// right-hand side's 3 plus the apply's 5.  b and b_prev are not written.
template <class T>
int enqueue_resid_init(fewha_handle* H, const Desc<T>& d, const T* s, T* c, cudaStream_t st, bool defer,
                       T* p0 = nullptr, T* phi_out = nullptr) {
    T* phi = phi_out ? phi_out : static_cast<T*>(H->phi);
    T* u = static_cast<T*>(H->u);
    int rc;
    ClArgs<T> a = cl_args<T>(H, c, phi);
    a.zero_piston = 1;
    if ((rc = launch_inv<T, 0>(H, d, a, st))) return rc;
    if ((rc = launch_proj<T>(H, d, phi, st))) return rc;
    if ((rc = launch_csensor<T, SSRC_RESID>(H, d, s, u, st))) return rc;
    if ((rc = launch_projT<T>(H, d, u, st))) return rc;
    ClArgs<T> b = cl_args<T>(H, u, static_cast<T*>(H->q));
    b.pin = c;
    b.iter = PQ_SCRATCH_SLOT;
    b.zero_piston = 1;
    b.vr = static_cast<T*>(H->r);
    b.vz = static_cast<T*>(H->z);
    b.vp = p0 ? p0 : static_cast<T*>(H->p);
    b.vj = static_cast<const T*>(H->Jinv);
    b.rzslot = 0;
    b.rzp = H->rzpart;
    b.defer_total = defer ? 1 : 0;
    return launch_fwd<T, LSRC_NODES, LDST_RESID_INIT>(H, d, b, st);
}

template <class T>
int enqueue_rhs(fewha_handle* H, const Desc<T>& d, const T* s, T* bout, cudaStream_t st) {
    T* u = static_cast<T*>(H->u);
    int rc;
    if ((rc = launch_csensor<T, SSRC_SLOPES>(H, d, s, u, st))) return rc;
    if ((rc = launch_projT<T>(H, d, u, st))) return rc;
    ClArgs<T> a = cl_args<T>(H, u, bout);
    a.zero_piston = 1;
    return launch_fwd<T, LSRC_NODES, LDST_COEF>(H, d, a, st);
}

int vec_grid(const fewha_handle* H) { return H->npart; }

template <class T, int PHASE>
int launch_vec(fewha_handle* H, int n, const VecArgs<T>& v, cudaStream_t st) {
    if (recorder<T>()) {
        record<T>(PHASE == V_INIT ? BK_VEC_INIT : PHASE == V_INIT_WARM ? BK_VEC_WARM : BK_VEC_UPDATE).va = v;
        return FEWHA_OK;
    }
    CK(launch_k(H, k_vec<T, PHASE>, dim3(vec_grid(H)), dim3(PBLK), 0, st, n, v), "k_vec launch");
    return FEWHA_OK;
}

template <class T>
int launch_fit(fewha_handle* H, const Desc<T>& d, const T* phi, T* a_prev, T* dm, int gain, cudaStream_t st,
               T* a_old = nullptr, const T* cpist = nullptr) {
    if (recorder<T>()) {
        if (gain == 2) return fail(H, FEWHA_ERR_INVALID_ARG, "closed-loop frames are not batched");
        record<T>(BK_FIT).fa = FitArgs<T>{phi, a_prev, dm, gain, cpist};
        return FEWHA_OK;
    }
    CK(launch_k(H, k_fit<T>, dim3((d.n_act + PBLK - 1) / PBLK), dim3(PBLK), 0, st, d, phi, a_prev, dm, gain,
                a_old, cpist),
       "k_fit launch");
    return FEWHA_OK;
}

// Pseudo-open-loop slopes s_pol = s + Gamma P_DM a^(i-1) (Algorithm 1, closed loop).
template <class T>
int launch_pol(fewha_handle* H, const Desc<T>& d, const T* s, T* out, cudaStream_t st) {
    if (recorder<T>()) return fail(H, FEWHA_ERR_INVALID_ARG, "closed-loop frames are not batched");
    PolArgs<T> p{s, static_cast<const T*>(H->a_old), out, static_cast<T*>(H->dm_nodes), H->qi0y, H->qi0x,
                 static_cast<const T*>(H->qfy), static_cast<const T*>(H->qfx)};
    CK(launch_k(H, k_dmnodes<T>, dim3((d.n_nodes + PBLK - 1) / PBLK), dim3(PBLK), 0, st, d, p),
       "k_dmnodes launch");
    int gx = 1;
    for (const WfsInfo& W : H->setup.G)
        gx = std::max(gx, W.nb == 1 ? (W.N * W.N + POLBLK - 1) / POLBLK : W.n_sub * W.n_sub);
    CK(launch_k(H, k_pol<T>, dim3(gx, d.n_wfs), dim3(POLBLK), 0, st, d, p), "k_pol launch");
    return FEWHA_OK;
}

// `iters` PCG iterations on M c = b (b in H->b), r0 explicit or warm.
// With s_resid (the explicit residual, single instances), r0 comes from the slopes'
// residual chain (enqueue_resid_init) and b is not formed.
template <class T>
int enqueue_pcg(fewha_handle* H, const Desc<T>& d, T* c, int iters, bool warm, cudaStream_t st,
                const T* s_resid = nullptr, bool carry = false) {
    // carry (with s_resid): the layers of c are carried through the iterations in H->phic
    // (W^T c without the full layers' pistons; the fit adds them), so the fit needs no
    // inverse transform
    T* phic = (carry && s_resid) ? static_cast<T*>(H->phic) : nullptr;
    int rc;
    // the initial residual's vector step fused into the forward kernel (single instances; the
    // batched frame keeps the separate vector kernel).  The iterations' CG updates stay in
    // their own kernel: fused behind a grid-wide wait for the p.q total (a cooperative
    // launch) they measured slower on GB300 than the separate launch.
    //
    // Dot totals are deferred to their consumers: no kernel of an iteration waits for a
    // grid-wide arrival count.  p.q of iteration k is totalled by the CG update of k; r.z of
    // slot k (the initial residual's for k = 0, else the update of k - 1) by the inverse
    // kernel that starts iteration k, which needs it for beta.  Every total still reaches
    // its slot (rztot[iters] through the last update's own arrival count).
    if (!recorder<T>()) {
        const bool defer = iters > 0;
        if (warm) {
            if ((rc = launch_vec<T, V_INIT_WARM>(H, d.n_c, vec_args<T>(H, c, 0), st))) return rc;
        } else if (s_resid) {
            if ((rc = enqueue_resid_init<T>(H, d, s_resid, c, st, defer, nullptr, phic))) return rc;
        } else {
            if ((rc = enqueue_apply_init<T>(H, d, c, st, defer))) return rc;
        }
        T* p = static_cast<T*>(H->p);
        for (int k = 0; k < iters; ++k) {
            Defer df;
            df.pq = true;
            if (k > 0) {
                df.rz_parts = H->rzpart + static_cast<size_t>(k) * H->npart;
                df.rz_cnt = H->npart;
                df.rz_slot = k;
            } else if (!warm) {
                df.rz_parts = H->rzpart;
                df.rz_cnt = d.n_layers * CL;
                df.rz_slot = 0;
            }
            if ((rc = enqueue_apply<T>(H, d, p, static_cast<T*>(H->q), k, k > 0, st, df))) return rc;
            VecArgs<T> v = vec_args<T>(H, c, k);
            v.pq_cnt = d.n_layers * CL;
            v.defer_rz = k + 1 < iters ? 1 : 0;
            v.phic = phic;
            v.phip = static_cast<const T*>(H->phi);
            if ((rc = launch_vec<T, V_UPDATE>(H, d.n_c, v, st))) return rc;
        }
        return FEWHA_OK;
    }
    if (warm) {
        if ((rc = launch_vec<T, V_INIT_WARM>(H, d.n_c, vec_args<T>(H, c, 0), st))) return rc;
    } else if (s_resid) {
        if ((rc = enqueue_resid_init<T>(H, d, s_resid, c, st, false, nullptr, phic))) return rc;
    } else {
        if ((rc = enqueue_apply<T>(H, d, c, static_cast<T*>(H->q), PQ_SCRATCH_SLOT, false, st))) return rc;
        if ((rc = launch_vec<T, V_INIT>(H, d.n_c, vec_args<T>(H, c, 0), st))) return rc;
    }
    T* p = static_cast<T*>(H->p);
    for (int k = 0; k < iters; ++k) {
        if ((rc = enqueue_apply<T>(H, d, p, static_cast<T*>(H->q), k, k > 0, st))) return rc;
        VecArgs<T> v = vec_args<T>(H, c, k);
        v.phic = phic;
        v.phip = static_cast<const T*>(H->phi);
        if ((rc = launch_vec<T, V_UPDATE>(H, d.n_c, v, st))) return rc;
    }
    return FEWHA_OK;
}

template <class T, int PHASE>
int launch_aug(fewha_handle* H, int n, const VecArgs<T>& v, const AugArgs<T>& a, cudaStream_t st) {
    if (recorder<T>()) return fail(H, FEWHA_ERR_INVALID_ARG, "augmented PCG frames are not batched");
    CK(launch_k(H, k_aug<T, PHASE>, dim3(vec_grid(H)), dim3(PBLK), 0, st, n, v, a), "k_aug launch");
    return FEWHA_OK;
}

// Device arrays of the augmented PCG, allocated on first use (never inside a capture).
int ensure_aug(fewha_handle* H) {
    if (H->Pd[0]) return FEWHA_OK;
    const size_t ld = (static_cast<size_t>(H->setup.n_c) + 63) & ~static_cast<size_t>(63);
    int rc;
    for (int s = 0; s < 2; ++s)
        if ((rc = talloc(H, &H->Pd[s], AUG_MAX * ld)) || (rc = talloc(H, &H->Qd[s], AUG_MAX * ld)) ||
            (rc = dalloc(H, &H->pqd[s], AUG_MAX)))
            return rc;
    if ((rc = dalloc(H, &H->augpart, static_cast<size_t>(AUG_MAX) * NPART_MAX)) ||
        (rc = dalloc(H, &H->augtot, 2 * AUG_MAX)))
        return rc;
    H->aug_ld = ld;
    return FEWHA_OK;
}

// Augmented PCG of Algorithm 1 (Sec. 3.4): `iters` iterations on M c = b whose directions
// and images go to set `set`, augmented by the `m` directions of the other set (the
// previous frame's; m = 0 on the first frame).  Each direction is formed by a vector
// kernel and the apply runs on it without the fused update.
template <class T>
int enqueue_pcg_aug(fewha_handle* H, const Desc<T>& d, T* c, int iters, bool warm, int set, int m,
                    cudaStream_t st, const T* s_resid = nullptr) {
    const size_t ld = H->aug_ld;
    T* Pn = static_cast<T*>(H->Pd[set]);
    T* Qn = static_cast<T*>(H->Qd[set]);
    AugArgs<T> a;
    a.P = static_cast<const T*>(H->Pd[1 - set]);
    a.Q = static_cast<const T*>(H->Qd[1 - set]);
    a.pq = H->pqd[1 - set];
    a.pqnew = H->pqd[set];
    a.part = H->augpart;
    a.tot = H->augtot;
    a.ld = static_cast<long long>(ld);
    a.m = m;
    a.mu_next = 0;
    int rc;
    VecArgs<T> v = vec_args<T>(H, c, 0);
    if (!warm && s_resid) {
        // r0 from the slopes' residual chain (its vector step writes z0 and p0 = z0, the
        // first direction of this set when there are no previous directions); with
        // previous directions, their p_j.r0, then the corrected start
        if ((rc = enqueue_resid_init<T>(H, d, s_resid, c, st, false, m > 0 ? nullptr : Pn))) return rc;
        if (m > 0 && ((rc = launch_aug<T, V_AUG_R0_RESID>(H, d.n_c, v, a, st)) ||
                      (rc = launch_aug<T, V_AUG_INIT>(H, d.n_c, v, a, st))))
            return rc;
    } else {
        if (!warm && (rc = enqueue_apply<T>(H, d, c, static_cast<T*>(H->q), PQ_SCRATCH_SLOT, false, st)))
            return rc;
        if (m > 0) {
            rc = warm ? launch_aug<T, V_AUG_R0_WARM>(H, d.n_c, v, a, st) : launch_aug<T, V_AUG_R0>(H, d.n_c, v, a, st);
            if (rc || (rc = launch_aug<T, V_AUG_INIT>(H, d.n_c, v, a, st))) return rc;
        } else {
            v.p = Pn;                            // p_0 = z_0
            rc = warm ? launch_vec<T, V_INIT_WARM>(H, d.n_c, v, st) : launch_vec<T, V_INIT>(H, d.n_c, v, st);
            if (rc) return rc;
        }
    }
    // Deferred totals (as in the plain PCG, single instances): the forward kernels leave p.q
    // to the CG update; the update of iteration k leaves r.z and its q_j.z dots to the
    // inverse kernel of iteration k + 1 (all but the last iteration's, whose r.z is totalled
    // by its own arrival count)
    const bool defer = !recorder<T>();
    for (int k = 0; k < iters; ++k) {
        T* pk = Pn + k * ld;
        T* qk = Qn + k * ld;
        v = vec_args<T>(H, c, k);
        Defer df;
        df.pq = defer;
        if (defer && k > 0) {
            df.rz_parts = H->rzpart + static_cast<size_t>(k) * H->npart;
            df.rz_cnt = H->npart;
            df.rz_slot = k;
        }
        if (k > 0 || m > 0) {
            // p_k = z_k + beta p_(k-1) - P mu, fused into the apply's inverse kernel
            rc = enqueue_apply_aug<T>(H, d, k > 0 ? Pn + (k - 1) * ld : nullptr, pk, static_cast<const T*>(H->z), qk,
                                      k, a, st, df, (defer && k > 0) ? H->npart : 0);
        } else {
            rc = enqueue_apply<T>(H, d, pk, qk, k, false, st, df);   // p_0 = z_0 (no directions)
        }
        if (rc) return rc;
        v.p = pk;
        v.q = qk;
        v.pq_cnt = defer ? d.n_layers * CL : 0;
        v.defer_rz = (defer && k + 1 < iters) ? 1 : 0;
        a.mu_next = (m > 0 && k + 1 < iters) ? 1 : 0;
        if ((rc = launch_aug<T, V_UPDATE_AUG>(H, d.n_c, v, a, st))) return rc;
    }
    return FEWHA_OK;
}

// carried: the layers of c are in H->phic already (enqueue_pcg's carry), without the full
// layers' pistons, which the fit adds from c
template <class T>
int enqueue_fit(fewha_handle* H, const Desc<T>& d, const T* c, T* dm, bool gain, cudaStream_t st,
                bool carried = false) {
    T* phi = static_cast<T*>(carried ? H->phic : H->phi);
    int rc;
    if (!carried && (rc = launch_inv<T, 0>(H, d, cl_args<T>(H, c, phi), st))) return rc;
    const bool closed = gain && (H->params.flags & FEWHA_FLAG_CLOSED_LOOP);
    return launch_fit<T>(H, d, phi, static_cast<T*>(H->a_prev), dm, closed ? 2 : (gain ? 1 : 0), st,
                         static_cast<T*>(H->a_old), carried ? c : nullptr);
}

template <class K>
int allow_smem(fewha_handle* H, K kernel, size_t need);

// Set-up of the persistent frame: its shared memory (the largest of the stages' bodies) and
// its clusters, at least one per layer and per sensor, up to one CTA per (sensor, layer)
// pair, no more than can be co-resident (cooperative launch).
template <class T>
int persistent_setup(fewha_handle* H) {
    if (H->pers_ncl) return FEWHA_OK;
    const HostSetup& s = H->setup;
    const int nl = static_cast<int>(s.L.size()), nw = static_cast<int>(s.G.size());
    H->smem_frame = std::max({H->smem_fwd, H->smem_inv, H->smem_sen, H->smem_proj, H->smem_projT});
    int rc;
    if ((rc = allow_smem(H, k_frame<T>, H->smem_frame))) return rc;
    const int need = std::max(nl, nw), want = std::max(need, (nl * nw + CL - 1) / CL);
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(CL, want);
    q.blockDim = dim3(cblk<T>());
    q.dynamicSmemBytes = H->smem_frame;
    int fit = 0;
    CK(cudaOccupancyMaxActiveClusters(&fit, k_frame<T>, &q), "persistent frame occupancy");
    if (fit < need) return fail(H, FEWHA_ERR_LIMIT, "persistent frame: too few co-resident clusters");
    H->pers_ncl = std::min(want, fit);
    return FEWHA_OK;
}

// One frame of Algorithm 1 as the persistent kernel (see fewha_persist.cuh).
template <class T>
int enqueue_persistent(fewha_handle* H, const T* s, T* c, T* dm, bool warm, cudaStream_t st) {
    const Desc<T> d = make_desc<T>(H);
    const int ncl = H->pers_ncl, nctas = ncl * CL;
    FrameArgs<T> f;
    f.s = s;
    f.c = c;
    f.dm = dm;
    f.a_prev = static_cast<T*>(H->a_prev);
    f.b = static_cast<T*>(H->b);
    f.phi = static_cast<T*>(H->phi);
    f.u = static_cast<T*>(H->u);
    f.q = static_cast<T*>(H->q);
    f.v = vec_args<T>(H, c, 0);
    f.v.pcg.npart = nctas;
    f.status = H->status;
    f.iters = H->params.iters;
    f.warm = warm ? 1 : 0;
    f.apply_gain = 1;
    f.pq_scratch = PQ_SCRATCH_SLOT;
    const GridSync g{H->gbar, H->gbar + 1, H->status, H->wait_limit, H->wait_extra, static_cast<unsigned>(nctas)};
    CK(cudaMemsetAsync(H->gbar, 0, 2 * sizeof(unsigned), st), "persistent frame barrier");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, ncl);
    cfg.blockDim = dim3(cblk<T>());
    cfg.dynamicSmemBytes = H->smem_frame;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, k_frame<T>, d, H->lay_fwd, H->lay_inv, H->lay_sen, pair_bufs<T>(H), f, g),
       "k_frame launch");
    return FEWHA_OK;
}

// One frame of Algorithm 1 (open loop).
// (With FEWHA_FLAG_AUGMENTED the PCG is the augmented one; its directions go to set
// H->aug_set, augmented by the H->aug_m directions of the other set.)
template <class T>
int enqueue_frame(fewha_handle* H, const T* s, T* c, T* dm, bool warm, cudaStream_t st) {
    if ((H->params.flags & FEWHA_FLAG_PERSISTENT) && !recorder<T>())
        return enqueue_persistent<T>(H, s, c, dm, warm, st);
    const Desc<T> d = make_desc<T>(H);
    int rc;
    if (H->params.flags & FEWHA_FLAG_CLOSED_LOOP) {
        // closed loop: the slopes are residual slopes; form the pseudo-open-loop slopes
        T* sp = static_cast<T*>(H->s_pol);
        if ((rc = launch_pol<T>(H, d, s, sp, st))) return rc;
        s = sp;
    }
    // the explicit-residual frame (plain or augmented, single or batched) forms r0 from the
    // slopes' residual (no b); the warm recurrence keeps b (its b_prev) and forms it first
    const bool resid = !warm && !(H->params.flags & FEWHA_FLAG_WARM_RESIDUAL);
    if (!resid && (rc = enqueue_rhs<T>(H, d, s, static_cast<T*>(H->b), st))) return rc;
    // the plain frame with the residual chain also carries the layers of c through its
    // iterations, so that its fit needs no inverse transform
    const bool carry = resid && !(H->params.flags & FEWHA_FLAG_AUGMENTED);
    if (H->params.flags & FEWHA_FLAG_AUGMENTED)
        rc = enqueue_pcg_aug<T>(H, d, c, H->params.iters, warm, H->aug_set, H->aug_m, st, resid ? s : nullptr);
    else
        rc = enqueue_pcg<T>(H, d, c, H->params.iters, warm, st, resid ? s : nullptr, carry);
    if (rc) return rc;
    return enqueue_fit<T>(H, d, c, dm, true, st, carry);
}

void drop_graph(fewha_handle* H) {
    for (auto& g : H->gexec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    for (auto& g : H->gaug) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    H->g_s = nullptr;
    H->g_x = nullptr;
    H->g_dm = nullptr;
}

template <class T>
int run_frame(fewha_handle* H, const T* s, T* c, T* dm, cudaStream_t st) {
    // the warm recurrence, unless a periodic explicit refresh is due
    const bool warm = (H->params.flags & FEWHA_FLAG_WARM_RESIDUAL) && H->have_prev &&
                      !(H->params.warm_refresh > 0 && H->warm_run >= H->params.warm_refresh);
    const bool aug = (H->params.flags & FEWHA_FLAG_AUGMENTED) != 0;
    int rc;
    if (aug && (rc = ensure_aug(H))) return rc;
    if ((H->params.flags & FEWHA_FLAG_PERSISTENT) && (rc = persistent_setup<T>(H))) return rc;
    if (H->params.flags & FEWHA_FLAG_GRAPH) {
        if (H->g_s != s || H->g_x != c || H->g_dm != dm || (aug && H->g_warm != warm)) drop_graph(H);
        // one graph per form: plain per initial residual (explicit, warm), or augmented per
        // (direction set, directions present)
        cudaGraphExec_t* gx = aug ? &H->gaug[2 * H->aug_set + (H->aug_m > 0 ? 1 : 0)] : &H->gexec[warm ? 1 : 0];
        if (!*gx) {
            CK(cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            rc = enqueue_frame<T>(H, s, c, dm, warm, H->cap_stream);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(H->cap_stream, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return cuda_fail(H, e, "end capture");
            e = cudaGraphInstantiate(gx, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                *gx = nullptr;
                return cuda_fail(H, e, "graph instantiate");
            }
            H->g_s = s;
            H->g_x = c;
            H->g_dm = dm;
            H->g_warm = warm;
        }
        CK(cudaGraphLaunch(*gx, st), "graph launch");
    } else {
        if ((rc = enqueue_frame<T>(H, s, c, dm, warm, st))) return rc;
    }
    H->have_prev = true;
    H->warm_run = warm ? H->warm_run + 1 : 0;
    if (aug) {
        H->aug_m = H->params.iters;
        H->aug_set = 1 - H->aug_set;
    }
    return FEWHA_OK;
}

// D, the exact data diagonal (GPU) and J^-1 for the current parameters.
template <class T>
int compute_diagonals(fewha_handle* H) {
    std::vector<double> D;
    prior_diag(H->setup, H->weights, H->params.r0, H->params.L0, D);
    if (upload(H, H->D64, D)) return FEWHA_ERR_CUDA;
    // D is constant per (layer, level): one value per level for the forward kernel, read at
    // row 0, column n / 2^k (detail level k) and at (0, 0) (the LL band)
    HostSetup& su = H->setup;
    su.dlev.assign(static_cast<size_t>(MAXL) * (MAXLEV + 1), 0.0);
    for (size_t l = 0; l < su.L.size(); ++l) {
        const LayerInfo& L = su.L[l];
        for (int k = 1; k <= L.levels; ++k) su.dlev[l * (MAXLEV + 1) + k] = D[L.off + (L.n >> k)];
        su.dlev[l * (MAXLEV + 1) + L.levels + 1] = D[L.off];
    }
    const Desc<T> d = make_desc<T>(H);
    DiagArgs a{H->basis, H->basis_off, H->pfy64, H->pfx64, H->Jdata};
    k_jdiag<T><<<(d.n_c + 3) / 4, 128>>>(d, a);
    CK(cudaGetLastError(), "k_jdiag launch");
    k_jfinish<T><<<(d.n_c + 255) / 256, 256>>>(d.n_c, H->Jdata, H->D64, H->params.alpha,
                                                H->params.tau, static_cast<T*>(H->Jinv),
                                                static_cast<T*>(H->D), H->J64);
    CK(cudaGetLastError(), "k_jfinish launch");
    CK(cudaDeviceSynchronize(), "diagonal set-up");
    return FEWHA_OK;
}

template <class T>
int setup_tables(fewha_handle* H) {
    const HostSetup& s = H->setup;
    int rc = 0;
    auto conv = [&](void* dst, const std::vector<double>& src) -> int {
        if (src.empty()) return FEWHA_OK;
        std::vector<T> tmp(src.begin(), src.end());
        CK(cudaMemcpy(dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice), "table upload");
        return FEWHA_OK;
    };
    if ((rc = conv(H->pfy, s.pfy)) || (rc = conv(H->pfx, s.pfx)) || (rc = conv(H->dfw, s.dfw))) return rc;
    // wavelet taps
    float h32[6], g32[6];
    for (int t = 0; t < 6; ++t) {
        h32[t] = static_cast<float>(s.taps_h[t]);
        g32[t] = static_cast<float>(s.taps_g[t]);
    }
    CK(cudaMemcpyToSymbol(c_h32, h32, sizeof(h32)), "taps");
    CK(cudaMemcpyToSymbol(c_g32, g32, sizeof(g32)), "taps");
    CK(cudaMemcpyToSymbol(c_h64, s.taps_h, sizeof(s.taps_h)), "taps");
    CK(cudaMemcpyToSymbol(c_g64, s.taps_g, sizeof(s.taps_g)), "taps");
    return compute_diagonals<T>(H);
}

// Let `kernel` use all dynamic shared memory left beside its static shared memory, and
// check that `need` bytes fit.
template <class K>
int allow_smem(fewha_handle* H, K kernel, size_t need) {
    cudaFuncAttributes fa;
    CK(cudaFuncGetAttributes(&fa, kernel), "function attributes");
    const int avail = 227 * 1024 - static_cast<int>(fa.sharedSizeBytes);
    if (need > static_cast<size_t>(avail))
        return fail(H, FEWHA_ERR_LIMIT, "cluster shared-memory tile above the per-CTA limit");
    CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, avail), "smem attr");
    return FEWHA_OK;
}

template <class T>
int set_smem_limits(fewha_handle* H) {
    const int maxsm = 227 * 1024;
    if (H->smem_layer > static_cast<size_t>(maxsm) || H->smem_sensor > static_cast<size_t>(maxsm))
        return fail(H, FEWHA_ERR_LIMIT, "shared-memory tile above 227 KB");
#define SETL(S, D, P) \
    CK(cudaFuncSetAttribute(k_layer<T, S, D, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm), "smem attr")
    SETL(LSRC_COEF, LDST_PHI, false);
    SETL(LSRC_COEF, LDST_PHI, true);
    SETL(LSRC_NODES, LDST_APPLY, false);
    SETL(LSRC_NODES, LDST_COEF, false);
    SETL(LSRC_NODES, LDST_PHI, false);
    SETL(LSRC_PHI, LDST_COEF, false);
    SETL(LSRC_DM, LDST_COEF, false);
#undef SETL
#define SETS(S, W, D) \
    CK(cudaFuncSetAttribute(k_sensor<T, S, W, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm), "smem attr")
    SETS(SSRC_PHI, true, SDST_ADJ);
    SETS(SSRC_SLOPES, true, SDST_ADJ);
    SETS(SSRC_PHI, false, SDST_NODES);
    SETS(SSRC_NODES, false, SDST_SLOPES);
    SETS(SSRC_SLOPES, false, SDST_ADJ);
    SETS(SSRC_SLOPES, true, SDST_SLOPES);
    SETS(SSRC_PHI, false, SDST_SLOPES);
#undef SETS
    if (H->smem_fwd > static_cast<size_t>(maxsm) || H->smem_inv > static_cast<size_t>(maxsm) ||
        H->smem_sen > static_cast<size_t>(maxsm))
        return fail(H, FEWHA_ERR_LIMIT, "cluster shared-memory tile above 227 KB");
    int rc = 0;
    if ((rc = allow_smem(H, k_cl_fwd<T, LSRC_NODES, LDST_APPLY>, H->smem_fwd)) ||
        (rc = allow_smem(H, k_cl_fwd<T, LSRC_NODES, LDST_COEF>, H->smem_fwd)) ||
        (rc = allow_smem(H, k_cl_fwd<T, LSRC_NODES, LDST_APPLY_INIT>, H->smem_fwd)) ||
        (rc = allow_smem(H, k_cl_fwd<T, LSRC_NODES, LDST_RESID_INIT>, H->smem_fwd)) ||
        (rc = allow_smem(H, k_cl_inv<T, 0>, H->smem_inv)) ||
        (rc = allow_smem(H, k_cl_inv<T, 1>, H->smem_inv)) ||
        (rc = allow_smem(H, k_cl_inv<T, 2>, H->smem_inv)) ||
        (rc = allow_smem(H, k_cl_sensor<T, SSRC_PHI>, H->smem_sen)) ||
        (rc = allow_smem(H, k_cl_sensor<T, SSRC_SLOPES>, H->smem_sen)) ||
        (rc = allow_smem(H, k_cl_sensor<T, SSRC_RESID>, H->smem_sen)) ||
        (rc = allow_smem(H, k_proj<T>, H->smem_proj)) || (rc = allow_smem(H, k_projT<T, 4>, H->smem_projT)) ||
        (rc = allow_smem(H, k_projT<T, KMAX>, H->smem_projT)))
        return rc;
    return FEWHA_OK;
}

// One periodic db3 step of the host (the same rule as the kernels' dwt_run): analysis of
// the m values x[0], x[st], ... into [a | d], or synthesis of [a | d] back.
// Whether some layer's coarse levels end with the three tail levels (Desc::tailop).
bool tail_used(const HostSetup& s) {
    for (const auto& L : s.L)
        if (L.levels >= 4 && (L.n >> (L.levels - 1)) == 2) return true;
    return false;
}

// Shared-memory layouts of the cluster kernels: the largest band over all layers and
// sensors, element counts in T units after a fixed header; every region starts on a
// 16-byte boundary (cp.async targets).
int round4(int x) { return (x + 3) & ~3; }

template <class T>
int cluster_layouts(fewha_handle* H) {
    const HostSetup& s = H->setup;
    constexpr int V = vec16<T>();
    int ybuf = 0, cbuf = 0, lbuf = 0, kmax = 0;
    for (size_t l = 0; l < s.L.size(); ++l) {
        const int n = s.L[l].n, rb = n >= CL ? n / CL : 1, h = n / 2;
        ybuf = std::max(ybuf, rb * (n + 1));
        cbuf = std::max(cbuf, n * (rb + 1));
        if (s.L[l].levels >= 2) lbuf = std::max(lbuf, h * (h + 1));
        for (size_t g = 0; g < s.G.size(); ++g) {
            const int rbk = static_cast<int>((g * MAXL + l) * MAXN);
            for (int i = 0; i < n; ++i) {
                kmax = std::max(kmax, s.ry_hi[rbk + i] - s.ry_lo[rbk + i]);
                kmax = std::max(kmax, s.rx_hi[rbk + i] - s.rx_lo[rbk + i]);
            }
        }
    }
    if (kmax > KMAX) return fail(H, FEWHA_ERR_LIMIT, "more than 8 aperture rows touch one layer row");
    H->kmax = kmax;
    ybuf = round4(ybuf);
    cbuf = round4(cbuf);
    lbuf = round4(lbuf);
    const size_t hdr_cl = RED_DBL * sizeof(double);
    ClLayout f{};
    f.ybuf = 0;
    f.cbuf = ybuf;
    f.lbuf = ybuf + cbuf;
    f.total = f.lbuf + lbuf;
    H->lay_fwd = f;
    H->smem_fwd = hdr_cl + static_cast<size_t>(f.total) * sizeof(T);
    ClLayout v{};
    v.ybuf = 0;
    v.cbuf = ybuf;
    v.lbuf = ybuf + cbuf;
    v.stage = v.lbuf + lbuf;                               // p and z of the column band
    v.stage2 = v.stage + 2 * MAXN * (MAXN / CL);           // p and z of the LL quadrant
    v.total = v.stage2 + 2 * (MAXN / 2) * (MAXN / 2);
    // the tail operator of the coarse levels (the forward kernel's region is placed after
    // its staged band sums, space permitting)
    std::vector<double> tail = tail_used(s) ? tail_operator(s.taps_h, s.taps_g, TAIL_LD) : std::vector<double>();
    if (!tail.empty()) {
        v.tail = v.total;
        v.total += round4(TAIL_N);
        int rc0;
        if ((rc0 = talloc(H, &H->tailop, TAIL_N))) return rc0;
        const std::vector<T> tt(tail.begin(), tail.end());
        CK(cudaMemcpy(H->tailop, tt.data(), tt.size() * sizeof(T), cudaMemcpyHostToDevice), "tail operator");
    }
    H->lay_inv = v;
    H->smem_inv = hdr_cl + static_cast<size_t>(v.total) * sizeof(T);
    int Vn = 0, SXn = 0, halo = 0;
    for (size_t g = 0; g < s.G.size(); ++g) {
        const int N = s.G[g].N, sr = (N + CL - 1) / CL;
        Vn = std::max(Vn, (sr + 1) * (N + 1));
        SXn = std::max(SXn, sr * N);
        halo = std::max(halo, 2 * N + 2 * MAXCOARSE);
    }
    SensorLayout q{};
    q.phsub = 0;
    q.V = 0;
    q.SX = q.V + round4(Vn);
    q.SY = q.SX + round4(SXn);
    q.halo = q.SY + round4(SXn);
    q.total = q.halo + round4(halo);
    q.msk = q.total;                               // rows x N ints
    q.total += round4(SXn);
    H->lay_sen = q;
    const size_t hdr_s = (RED_DBL + 2 + 2 * MAXCOARSE) * sizeof(double) + (4 * MAXL + 4) * sizeof(int);
    H->smem_sen = hdr_s + static_cast<size_t>(q.total) * sizeof(T);
    // pair kernels: footprint boxes (16-byte aligned column supersets) and tile sizes
    std::vector<int> box(MAXG * MAXL * 4, 0);
    size_t proj = 0, projT = 0;
    int yslot = 4;
    for (size_t g = 0; g < s.G.size(); ++g) {
        const int N = s.G[g].N, NP = N + 1;
        for (size_t l = 0; l < s.L.size(); ++l) {
            const int tp = static_cast<int>((g * MAXL + l) * TAB);
            const int n = s.L[l].n;
            const int al = (n % V) == 0 ? V : 1;
            const int r0 = s.pi0y[tp + 0], rows = s.pi0y[tp + N] + 2 - r0;
            const int c0 = s.pi0x[tp + 0] & ~(al - 1);
            const int c1 = (s.pi0x[tp + N] + 2 + al - 1) & ~(al - 1);
            int* bx = &box[(g * MAXL + l) * 4];
            bx[0] = r0;
            bx[1] = rows;
            bx[2] = c0;
            bx[3] = c1 - c0;
            yslot = std::max(yslot, round4(rows * (c1 - c0)));
            proj = std::max(proj, static_cast<size_t>(round4(rows * (c1 - c0)) + rows * NP + 4 * NP + 4));
            projT = std::max(projT, static_cast<size_t>(round4(2 * V + NP * NP) + round4(NP * (c1 - c0)) +
                                                        (c1 - c0 + rows + 2) * (KMAX + 2) + 8));
        }
    }
    H->box_host = box;
    // adjoint-projection weights of every pair (see PairBufs::tw / ti), in T arithmetic
    {
        const int nl = static_cast<int>(s.L.size()), ng = static_cast<int>(s.G.size());
        std::vector<T> tw(static_cast<size_t>(ng) * nl * 2 * MAXN * KMAX, T(0));
        std::vector<int> ti(static_cast<size_t>(ng) * nl * 2 * MAXN * 2 + 16, 0);
        for (int g = 0; g < ng; ++g)
            for (int l = 0; l < nl; ++l) {
                const int pr = g * nl + l, n = s.L[l].n;
                const int tp = (g * MAXL + l) * TAB, rbk = (g * MAXL + l) * MAXN;
                const int* bx = &box[(g * MAXL + l) * 4];
                for (int q = 0; q < 2; ++q) {
                    const int cnt = q == 0 ? bx[3] : bx[1], base = q == 0 ? bx[2] : bx[0];
                    const std::vector<int>& lo = q == 0 ? s.rx_lo : s.ry_lo;
                    const std::vector<int>& hi = q == 0 ? s.rx_hi : s.ry_hi;
                    const std::vector<int>& i0 = q == 0 ? s.pi0x : s.pi0y;
                    const std::vector<double>& fw = q == 0 ? s.pfx : s.pfy;
                    for (int k = 0; k < cnt && k < MAXN; ++k) {
                        const int j = base + k;
                        int b0 = 0, c = 0;
                        if (j < n) {
                            b0 = lo[rbk + j];
                            c = hi[rbk + j] - b0;
                        }
                        int* e = &ti[((static_cast<size_t>(pr) * 2 + q) * MAXN + k) * 2];
                        e[0] = b0;
                        e[1] = c;
                        T* w = &tw[((static_cast<size_t>(pr) * 2 + q) * MAXN + k) * KMAX];
                        for (int m = 0; m < c && m < KMAX; ++m) {
                            const T f = static_cast<T>(fw[tp + b0 + m]);
                            w[m] = i0[tp + b0 + m] == j ? T(1) - f : f;
                        }
                    }
                }
            }
        int rc0;
        if ((rc0 = talloc(H, &H->ptw, tw.size())) || (rc0 = dalloc(H, &H->pti, ti.size()))) return rc0;
        CK(cudaMemcpy(H->ptw, tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice), "projection weights");
        if ((rc0 = upload(H, H->pti, ti))) return rc0;
    }
    // staged pair terms of the forward kernel's band: per layer and cluster rank, the
    // band's rows of every sensor's term, each run rounded to a 16-byte chunk
    bool aligned = true;
    int ystg = 0;
    for (size_t l = 0; l < s.L.size(); ++l) {
        const int n = s.L[l].n, rb = n >= CL ? n / CL : 1;
        for (int r = 0; r * rb < n && r < CL; ++r) {
            int need = 0;
            for (size_t g = 0; g < s.G.size(); ++g) {
                const int* bx = &box[(g * MAXL + l) * 4];
                aligned = aligned && (bx[2] % V) == 0 && (bx[3] % V) == 0 && (n % V) == 0;
                const int lo = std::max(r * rb, bx[0]), hi = std::min(r * rb + rb, bx[0] + bx[1]);
                if (hi > lo) need += ((hi - lo) * bx[3] + V - 1) & ~(V - 1);
            }
            ystg = std::max(ystg, need);
        }
    }
    // the batched kernels also hold their instance's descriptor in static shared memory
    const long long spare = 227LL * 1024 - static_cast<long long>(H->smem_fwd) -
                            static_cast<long long>(sizeof(Desc<T>)) - 2048;
    std::vector<int> ytab;
    // single precision reads the band's terms straight from L2 (one 16-byte group per thread
    // and sensor, every read in flight at once); double precision stages them in shared
    // memory (its threads own several groups each)
    const bool direct = aligned && ystg > 0 && sizeof(T) == 4;
    if (direct ||
        (aligned && ystg > 0 && static_cast<long long>(round4(ystg)) * static_cast<long long>(sizeof(T)) <= spare)) {
        if (direct) {
            H->lay_fwd.ydirect = 1;
        } else {
            H->lay_fwd.ystg = H->lay_fwd.total;
            H->lay_fwd.total += round4(ystg);
            H->smem_fwd += static_cast<size_t>(round4(ystg)) * sizeof(T);
        }
        // the run table (see PairBufs::ytab)
        const int nw = static_cast<int>(s.G.size());
        ytab.assign(s.L.size() * CL * nw * 8, 0);
        for (size_t l = 0; l < s.L.size(); ++l) {
            const int n = s.L[l].n, rb = n >= CL ? n / CL : 1;
            for (int r = 0; r < CL; ++r) {
                int so = 0;
                for (int g = 0; g < nw; ++g) {
                    const int* bx = &box[(g * MAXL + l) * 4];
                    const int lo = std::max(r * rb, bx[0]);
                    const int hi = std::max(lo, std::min(r * rb + rb, bx[0] + bx[1]));
                    int* e = &ytab[((l * CL + r) * nw + g) * 8];
                    e[0] = lo;
                    e[1] = hi;
                    e[2] = bx[2];
                    e[3] = bx[3];
                    e[4] = so;
                    e[5] = (g * static_cast<int>(s.L.size()) + static_cast<int>(l)) * yslot + (lo - bx[0]) * bx[3];
                    so += ((hi - lo) * bx[3] + V - 1) & ~(V - 1);
                }
            }
        }
    }
    if (H->tailop) {
        const long long room = 227LL * 1024 - static_cast<long long>(H->smem_fwd) -
                               static_cast<long long>(sizeof(Desc<T>)) - 2048;
        if (static_cast<long long>(round4(TAIL_N)) * static_cast<long long>(sizeof(T)) <= room) {
            H->lay_fwd.tail = H->lay_fwd.total;
            H->lay_fwd.total += round4(TAIL_N);
            H->smem_fwd += static_cast<size_t>(round4(TAIL_N)) * sizeof(T);
        }
    }
    // single precision: the leader of a layer's cluster stages the LL quadrant's epilogue
    // operands (p, b, J^-1) and forms the LL epilogue itself (ClLayout::lstage); it needs
    // 16-byte aligned quadrant rows in every coarse layer
    if (sizeof(T) == 4) {
        bool ok = true;
        for (const auto& L : s.L)
            if (L.levels >= 2) ok = ok && (L.n / 2) % V == 0 && L.n % V == 0 && L.off % V == 0;
        const int need = round4(3 * (MAXN / 2) * (MAXN / 2));
        const long long room = 227LL * 1024 - static_cast<long long>(H->smem_fwd) -
                               static_cast<long long>(sizeof(Desc<T>)) - 2048;
        if (ok && static_cast<long long>(need) * static_cast<long long>(sizeof(T)) <= room) {
            H->lay_fwd.lstage = H->lay_fwd.total;
            H->lay_fwd.total += need;
            H->smem_fwd += static_cast<size_t>(need) * sizeof(T);
        }
    }
    H->smem_proj = proj * sizeof(T);
    H->smem_projT = projT * sizeof(T);
    H->pvs = round4(s.max_N + 1);
    H->pvslot = (s.max_N + 1) * H->pvs;
    H->pyslot = yslot;
    int rc;
    const size_t pairs = s.G.size() * s.L.size();
    if (!ytab.empty() && ((rc = dalloc(H, &H->ytab, ytab.size())) || (rc = upload(H, H->ytab, ytab)))) return rc;
    if ((rc = dalloc(H, &H->box, box.size())) || (rc = upload(H, H->box, box)) ||
        (rc = talloc(H, &H->pairV, pairs * H->pvslot)) || (rc = talloc(H, &H->pairY, pairs * H->pyslot)))
        return rc;
    return FEWHA_OK;
}

void free_handle(fewha_handle* H) {
    if (!H) return;
    drop_graph(H);
    if (H->cap_stream) cudaStreamDestroy(H->cap_stream);
    for (void* p : H->allocs) cudaFree(p);
    delete H->lsf;
    delete H;
}

int check_params(const fewha_params* p, std::string& err) {
    if (!p) {
        err = "params is NULL";
        return FEWHA_ERR_INVALID_ARG;
    }
    if (p->precision != 32 && p->precision != 64) {
        err = "precision must be 32 or 64";
        return FEWHA_ERR_INVALID_ARG;
    }
    if (p->iters < 0 || p->iters > FEWHA_MAX_ITERS) {
        err = "iters out of range";
        return FEWHA_ERR_LIMIT;
    }
    if (p->warm_refresh < 0) {
        err = "warm_refresh must be >= 0";
        return FEWHA_ERR_INVALID_ARG;
    }
    if ((p->flags & FEWHA_FLAG_PERSISTENT) && (p->flags & (FEWHA_FLAG_AUGMENTED | FEWHA_FLAG_CLOSED_LOOP))) {
        err = "the persistent frame runs the plain open-loop PCG only";
        return FEWHA_ERR_INVALID_ARG;
    }
    if ((p->flags & FEWHA_FLAG_AUGMENTED) && p->iters > FEWHA_AUG_MAX_ITERS) {
        err = "augmented PCG keeps at most FEWHA_AUG_MAX_ITERS directions";
        return FEWHA_ERR_LIMIT;
    }
    if (!(p->alpha >= 0) || !(p->tau >= 0) || !(p->r0 > 0) || !(p->L0 > 0) || !(p->gain >= 0) ||
        !(p->gain <= 1) || !(p->alpha_eta >= 0) || !std::isfinite(p->alpha_eta)) {
        err = "alpha, tau, alpha_eta >= 0, r0, L0 > 0 and gain in [0, 1] required";
        return FEWHA_ERR_INVALID_ARG;
    }
    return FEWHA_OK;
}

template <class T>
int typed_create(fewha_handle* H) {
    const HostSetup& s = H->setup;
    int rc = 0;
    const size_t tab = static_cast<size_t>(MAXG) * MAXL * TAB;
    const size_t rng = static_cast<size_t>(MAXG) * MAXL * MAXN;
    const size_t dtab = static_cast<size_t>(MAXM) * MAXL * MAXNACT;
    const size_t drng = static_cast<size_t>(MAXM) * MAXL * MAXN;
    if ((rc = dalloc(H, &H->pi0y, tab)) || (rc = dalloc(H, &H->pi0x, tab)) ||
        (rc = dalloc(H, &H->pfy64, tab)) || (rc = dalloc(H, &H->pfx64, tab)) ||
        (rc = dalloc(H, &H->ry_lo, rng)) || (rc = dalloc(H, &H->ry_hi, rng)) ||
        (rc = dalloc(H, &H->rx_lo, rng)) || (rc = dalloc(H, &H->rx_hi, rng)) ||
        (rc = dalloc(H, &H->sidx, s.sidx.size())) || (rc = dalloc(H, &H->cidx, s.cidx.size() + 1)) ||
        (rc = dalloc(H, &H->di0, dtab)) || (rc = dalloc(H, &H->dr_lo, drng)) ||
        (rc = dalloc(H, &H->dr_hi, drng)) || (rc = dalloc(H, &H->basis_off, s.basis_off.size())) ||
        (rc = dalloc(H, &H->basis, s.basis.size())) || (rc = dalloc(H, &H->D64, s.n_c)) ||
        (rc = dalloc(H, &H->Jdata, s.n_c)) || (rc = dalloc(H, &H->J64, s.n_c)) ||
        (rc = dalloc(H, &H->rzpart, static_cast<size_t>(FEWHA_MAX_ITERS + 2) * NPART_MAX)) ||
        (rc = dalloc(H, &H->pqpart, static_cast<size_t>(FEWHA_MAX_ITERS + 2) * PQ_SLOTS)) ||
        (rc = dalloc(H, &H->rztot, static_cast<size_t>(FEWHA_MAX_ITERS + 2))) ||
        (rc = dalloc(H, &H->pqtot, static_cast<size_t>(FEWHA_MAX_ITERS + 2))) ||
        (rc = dalloc(H, &H->count, 2)) || (rc = dalloc(H, &H->status, 1)) || (rc = dalloc(H, &H->gbar, 4)) ||
        (rc = dalloc(H, &H->qi0y, s.qi0y.size())) || (rc = dalloc(H, &H->qi0x, s.qi0x.size())))
        return rc;
    if ((rc = talloc(H, &H->pfy, tab)) || (rc = talloc(H, &H->pfx, tab)) ||
        (rc = talloc(H, &H->dfw, dtab)) || (rc = talloc(H, &H->D, s.n_c)) ||
        (rc = talloc(H, &H->Jinv, s.n_c)) || (rc = talloc(H, &H->c, s.n_c)) ||
        (rc = talloc(H, &H->b, s.n_c)) || (rc = talloc(H, &H->b_prev, s.n_c)) ||
        (rc = talloc(H, &H->r, s.n_c)) || (rc = talloc(H, &H->z, s.n_c)) ||
        (rc = talloc(H, &H->p, s.n_c)) || (rc = talloc(H, &H->q, s.n_c)) ||
        (rc = talloc(H, &H->phi, s.n_c)) || (rc = talloc(H, &H->phic, s.n_c)) || (rc = talloc(H, &H->c_tmp, s.n_c)) ||
        (rc = talloc(H, &H->u, s.n_nodes)) || (rc = talloc(H, &H->a_prev, s.n_act)) ||
        (rc = talloc(H, &H->dm_tmp, s.n_act)) || (rc = talloc(H, &H->s_tmp, s.n_s)) ||
        (rc = talloc(H, &H->cgrad, s.n_c)) || (rc = talloc(H, &H->lam, s.n_c)) ||
        (rc = dalloc(H, &H->gdot, MAXL + 1)) || (rc = talloc(H, &H->qfy, s.qfy.size())) ||
        (rc = talloc(H, &H->qfx, s.qfx.size())) || (rc = talloc(H, &H->s_pol, s.n_s)) ||
        (rc = talloc(H, &H->a_old, s.n_act)) || (rc = talloc(H, &H->dm_nodes, s.n_nodes)))
        return rc;
    if ((rc = upload(H, H->pi0y, s.pi0y)) || (rc = upload(H, H->pi0x, s.pi0x)) ||
        (rc = upload(H, H->pfy64, s.pfy)) || (rc = upload(H, H->pfx64, s.pfx)) ||
        (rc = upload(H, H->ry_lo, s.ry_lo)) || (rc = upload(H, H->ry_hi, s.ry_hi)) ||
        (rc = upload(H, H->rx_lo, s.rx_lo)) || (rc = upload(H, H->rx_hi, s.rx_hi)) ||
        (rc = upload(H, H->sidx, s.sidx)) || (rc = upload(H, H->cidx, s.cidx)) ||
        (rc = upload(H, H->di0, s.di0)) || (rc = upload(H, H->dr_lo, s.dr_lo)) ||
        (rc = upload(H, H->dr_hi, s.dr_hi)) || (rc = upload(H, H->basis_off, s.basis_off)) ||
        (rc = upload(H, H->basis, s.basis)) || (rc = upload(H, H->qi0y, s.qi0y)) ||
        (rc = upload(H, H->qi0x, s.qi0x)) ||
        (rc = upload(H, static_cast<T*>(H->qfy), std::vector<T>(s.qfy.begin(), s.qfy.end()))) ||
        (rc = upload(H, static_cast<T*>(H->qfx), std::vector<T>(s.qfx.begin(), s.qfx.end()))))
        return rc;
    H->smem_layer = (2 * NWARP + 4) * sizeof(double) + static_cast<size_t>(s.max_n) * s.max_n * sizeof(T);
    H->smem_sensor = (2 * NWARP + 4 + 2 * MAXCOARSE) * sizeof(double) +
                     (static_cast<size_t>(s.max_N + 1) * (s.max_N + 1) + 2 * static_cast<size_t>(s.max_N) * s.max_N) * sizeof(T);
    if ((rc = cluster_layouts<T>(H))) return rc;
    if ((rc = set_smem_limits<T>(H))) return rc;
    return setup_tables<T>(H);
}

template <class T>
int check_type(fewha_handle* H) {
    if (!H) return FEWHA_ERR_INVALID_ARG;
    if (static_cast<int>(sizeof(T) * 8) != H->precision)
        return fail(H, FEWHA_ERR_INVALID_ARG, "element type does not match the handle's precision");
    return FEWHA_OK;
}

template <class T>
int reconstruct_dev(fewha_handle* H, const T* s, T* x, T* dm, void* stream) {
    int rc;
    if ((rc = check_type<T>(H))) return rc;
    if (!s || !dm) return fail(H, FEWHA_ERR_INVALID_ARG, "null slope or DM pointer");
    DeviceGuard g(H->device);
    return run_frame<T>(H, s, x ? x : static_cast<T*>(H->c), dm, static_cast<cudaStream_t>(stream));
}

// Enqueue one frame from and to host memory; *flag receives the non-finite status.
template <class T>
int enqueue_host_frame(fewha_handle* H, const T* hs, T* hdm, unsigned* flag, cudaStream_t st) {
    const HostSetup& s = H->setup;
    int rc;
    CK(cudaMemcpyAsync(H->s_tmp, hs, s.n_s * sizeof(T), cudaMemcpyHostToDevice, st), "slopes H2D");
    if ((rc = run_frame<T>(H, static_cast<const T*>(H->s_tmp), static_cast<T*>(H->c),
                           static_cast<T*>(H->dm_tmp), st)))
        return rc;
    CK(cudaMemcpyAsync(hdm, H->dm_tmp, s.n_act * sizeof(T), cudaMemcpyDeviceToHost, st), "DM D2H");
    CK(cudaMemcpyAsync(flag, H->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "status");
    return FEWHA_OK;
}

// After the stream has synchronised: clear a raised non-finite flag.
// The frame's status word: bit 0 non-finite slopes, bit 1 a persistent frame's wait ran out.
int clear_flag(fewha_handle* H, unsigned flag, cudaStream_t st) {
    if (!flag) return FEWHA_OK;
    cudaMemsetAsync(H->status, 0, sizeof(unsigned), st);
    cudaStreamSynchronize(st);
    if (flag & 2u) return fail(H, FEWHA_ERR_TIMEOUT, "a grid-wide wait of the persistent frame ran out");
    return fail(H, FEWHA_ERR_NONFINITE, "non-finite value in the input slopes");
}

template <class T>
int reconstruct_host(fewha_handle* H, const T* hs, T* hdm, void* stream) {
    int rc;
    if ((rc = check_type<T>(H))) return rc;
    if (!hs || !hdm) return fail(H, FEWHA_ERR_INVALID_ARG, "null host pointer");
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned flag = 0;
    if ((rc = enqueue_host_frame<T>(H, hs, hdm, &flag, st))) return rc;
    CK(cudaStreamSynchronize(st), "host frame");
    return clear_flag(H, flag, st);
}

// Frames released on a fixed period from host buffers; see fewha_run_loop.
template <class T>
int run_loop(fewha_handle* H, const T* hs, int n_frames, T* hdm, double period_us, float* wall_us,
             float* device_us, int* n_late, void* stream) {
    int rc;
    if ((rc = check_type<T>(H))) return rc;
    if (n_frames < 0 || (n_frames > 0 && (!hs || !hdm)) || !(period_us >= 0.0))
        return fail(H, FEWHA_ERR_INVALID_ARG, "bad frame count, host pointer or period");
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const HostSetup& s = H->setup;
    using clock = std::chrono::steady_clock;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(H, FEWHA_ERR_CUDA, "event");
    }
    int late = 0, first_bad = -1;
    rc = FEWHA_OK;
    const clock::time_point t0 = clock::now();
    clock::time_point prev_end = t0;
    for (int k = 0; k < n_frames && rc == FEWHA_OK; ++k) {
        const clock::time_point release =
            t0 + std::chrono::duration_cast<clock::duration>(std::chrono::duration<double, std::micro>(period_us * k));
        while (clock::now() < release) {
        }
        const clock::time_point start = std::max(release, prev_end);
        unsigned flag = 0;
        cudaEventRecord(e0, st);
        if ((rc = enqueue_host_frame<T>(H, hs + static_cast<size_t>(k) * s.n_s,
                                        hdm + static_cast<size_t>(k) * s.n_act, &flag, st)))
            break;
        cudaEventRecord(e1, st);
        const cudaError_t se = cudaStreamSynchronize(st);
        if (se != cudaSuccess) {
            rc = cuda_fail(H, se, "loop frame");
            break;
        }
        const clock::time_point end = clock::now();
        const int fr = clear_flag(H, flag, st);
        if (fr == FEWHA_ERR_TIMEOUT) {
            rc = fail(H, fr, "a grid-wide wait of the persistent frame ran out in frame " + std::to_string(k));
            break;
        }
        if (fr && first_bad < 0) first_bad = k;
        if (wall_us) wall_us[k] = static_cast<float>(std::chrono::duration<double, std::micro>(end - start).count());
        if (device_us) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            device_us[k] = 1e3f * ms;
        }
        if (period_us > 0.0 && end > release + std::chrono::duration_cast<clock::duration>(
                                                   std::chrono::duration<double, std::micro>(period_us)))
            ++late;
        prev_end = end;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_late) *n_late = late;
    if (rc) return rc;
    if (first_bad >= 0)
        return fail(H, FEWHA_ERR_NONFINITE, "non-finite value in the slopes of frame " + std::to_string(first_bad));
    return FEWHA_OK;
}

// ---------------------------------------------------------------- converged solve and gradients
// x = M^-1 b by PCG until sqrt(r.J^-1 r / b.J^-1 b) <= tol or max_iters, from x = 0 or
// (warm) from the x given.  The iterations run in chunks (the scalar slots hold
// FEWHA_MAX_ITERS + 2 values); between chunks the last two r.z totals are moved to slots
// 0 and 1 and the next chunk resumes at iteration 1, whose fused direction update
// p = z + beta p continues the same CG recurrence (no restart).  Uses the frame's work
// vectors (b, r, z, p, q, b_prev), so the warm residual is discarded.  Synchronous.
template <class T>
int solve_converged(fewha_handle* H, const T* b, T* x, bool warm, double tol, int max_iters, cudaStream_t st,
                    int* iters_out, double* rel_out) {
    const Desc<T> d = make_desc<T>(H);
    int rc;
    if (b != static_cast<const T*>(H->b))
        CK(cudaMemcpyAsync(H->b, b, d.n_c * sizeof(T), cudaMemcpyDeviceToDevice, st), "solve rhs");
    if (!warm) CK(cudaMemsetAsync(x, 0, d.n_c * sizeof(T), st), "solve start");
    k_wnorm<T><<<1, PBLK, 0, st>>>(d.n_c, static_cast<const T*>(H->b), d.Jinv, H->gdot + MAXL);
    CK(cudaGetLastError(), "k_wnorm launch");
    double rzb = 0.0, rz = 0.0;
    CK(cudaMemcpyAsync(&rzb, H->gdot + MAXL, sizeof(double), cudaMemcpyDeviceToHost, st), "solve norm");
    int done = 0;
    T* p = static_cast<T*>(H->p);
    T* q = static_cast<T*>(H->q);
    while (done < max_iters) {
        int last;                                // slot of the newest r.z total
        if (done == 0) {
            const int k = std::min(FEWHA_MAX_ITERS, max_iters);
            if ((rc = enqueue_pcg<T>(H, d, x, k, false, st))) return rc;
            done = k;
            last = k;
        } else {
            // resume: slots (K-1, K) -> (0, 1), then iterations 1 .. k of the recurrence
            CK(cudaMemcpyAsync(H->rztot, H->rztot + FEWHA_MAX_ITERS - 1, 2 * sizeof(double),
                               cudaMemcpyDeviceToDevice, st), "solve resume");
            const int k = std::min(FEWHA_MAX_ITERS - 1, max_iters - done);
            for (int j = 1; j <= k; ++j) {
                if ((rc = enqueue_apply<T>(H, d, p, q, j, true, st))) return rc;
                if ((rc = launch_vec<T, V_UPDATE>(H, d.n_c, vec_args<T>(H, x, j), st))) return rc;
            }
            done += k;
            last = k + 1;
        }
        CK(cudaMemcpyAsync(&rz, H->rztot + last, sizeof(double), cudaMemcpyDeviceToHost, st), "solve residual");
        CK(cudaStreamSynchronize(st), "solve residual");
        if (!(rzb > 0.0) || !(rz > 0.0) || std::sqrt(rz / rzb) <= tol) break;
        if (last != FEWHA_MAX_ITERS) break;      // the chunk was cut short by max_iters
    }
    if (max_iters == 0) CK(cudaStreamSynchronize(st), "solve");
    H->have_prev = false;
    if (iters_out) *iters_out = done;
    if (rel_out) *rel_out = rzb > 0.0 ? std::sqrt(std::max(rz, 0.0) / rzb) : 0.0;
    if (!std::isfinite(rz)) return fail(H, FEWHA_ERR_NONFINITE, "non-finite residual in the converged solve");
    return FEWHA_OK;
}

// Zero the piston coefficient (the constant function) of every full-depth layer of a
// coefficient vector.  Used before the slope map Gamma P W^T of a gradient: Gamma
// annihilates constants, so this changes nothing mathematically, but the adjoint vectors
// carry a large piston component (J^-1 of that coefficient is ~1 / (alpha D_LL)) whose
// rounding in phi would otherwise leak through the differences of Gamma.
template <class T>
int zero_pistons(fewha_handle* H, T* v, cudaStream_t st) {
    for (const LayerInfo& L : H->setup.L)
        if (L.full) CK(cudaMemsetAsync(v + L.off, 0, sizeof(T), st), "zero piston");
    return FEWHA_OK;
}

// The double-precision twin of a single-precision handle: the same geometry and
// parameters, no flags.  It computes the true residuals b - M x of the single-precision
// form's converged solves and holds their double iterates.
int twin_params(fewha_handle* H) {
    fewha_params p = H->params;
    p.precision = 64;
    p.flags = 0;
    const int rc = fewha_update_params(H->twin, &p, H->weights.data(), H->setup.wfs_sigma.data());
    if (rc) return fail(H, rc, std::string("double-precision twin: ") + fewha_last_error(H->twin));
    return FEWHA_OK;
}

int ensure_twin(fewha_handle* H) {
    if (H->twin) return FEWHA_OK;
    fewha_params p = H->params;
    p.precision = 64;
    p.flags = 0;
    std::vector<fewha_layer> layers = H->layers_in;
    for (size_t l = 0; l < layers.size(); ++l) layers[l].cn2_weight = H->weights[l];
    std::vector<fewha_wfs> wfs = H->wfs_in;
    for (size_t g = 0; g < wfs.size(); ++g) wfs[g].sigma = H->setup.wfs_sigma[g];
    fewha_handle* X = nullptr;
    const int rc = fewha_create(&H->tel_in, wfs.data(), static_cast<int>(wfs.size()), layers.data(),
                                static_cast<int>(layers.size()), H->dms_in.empty() ? nullptr : H->dms_in.data(),
                                static_cast<int>(H->dms_in.size()), &p, &X);
    if (rc) return fail(H, rc, std::string("double-precision twin: ") + fewha_create_error());
    H->twin = X;
    return FEWHA_OK;
}

// b^T J^-1 b of a double vector of the twin, on the host (synchronises).
int twin_wnorm(fewha_handle* H, fewha_handle* X, const double* v, double* out, cudaStream_t st) {
    k_wnorm<double><<<1, PBLK, 0, st>>>(X->setup.n_c, v, static_cast<const double*>(X->Jinv), X->gdot + MAXL);
    CK(cudaGetLastError(), "k_wnorm launch");
    CK(cudaMemcpyAsync(out, X->gdot + MAXL, sizeof(double), cudaMemcpyDeviceToHost, st), "norm");
    CK(cudaStreamSynchronize(st), "norm");
    return FEWHA_OK;
}

// Mixed-precision converged solve of the single-precision form: M x64 = b64 (double
// vectors of the twin X) to sqrt(r^T J^-1 r / b^T J^-1 b) <= tol with r = b - M x64 the
// TRUE residual in double.  One CG recurrence runs in float on H (its operators, its
// vector kernels) on a residual scaled to unit J^-1-norm; its iterate is an increment
// that is folded into x64 whenever the recurrence's residual has dropped tenfold (or the
// chunk ends at max_iters, or the recurrence's estimate says tol is met).  The true
// residual then replaces the recurrence's (reliable updates, k_refresh), and the search
// direction continues, rescaled.  The float operator is accurate to ~1e-7 relative, far
// inside the tenfold reduction, so the recurrence converges like the double one (about
// 1.5 times its iterations were measured on the 8 m geometry) while every step is a
// float step.  *iters_out counts float iterations.  Synchronous.
int reliable_solve(fewha_handle* H, fewha_handle* X, const double* b64, double* x64, bool warm, double tol,
                   int max_iters, cudaStream_t st, int* iters_out, double* rel_out) {
    constexpr double DELTA = 0.1;
    const Desc<float> d = make_desc<float>(H);
    const Desc<double> dx = make_desc<double>(X);
    const int n = d.n_c;
    double* r64 = static_cast<double*>(X->r);
    double* q64 = static_cast<double*>(X->q);
    float* x32 = static_cast<float*>(H->c_tmp);
    float* p = static_cast<float*>(H->p);
    float* q = static_cast<float*>(H->q);
    int rc;
    double bn2 = 0.0, rr2 = 0.0;
    if ((rc = twin_wnorm(H, X, b64, &bn2, st))) return rc;
    if (!warm) CK(cudaMemsetAsync(x64, 0, n * sizeof(double), st), "solve start");
    const int gl = std::min(4 * 152, (n + PBLK - 1) / PBLK);
    auto true_residual = [&]() -> int {
        int r2 = 0;
        if ((r2 = enqueue_apply<double>(X, dx, x64, q64, PQ_SCRATCH_SLOT, false, st))) return fail(H, r2, X->err);
        k_lin<double><<<gl, PBLK, 0, st>>>(n, 1.0, b64, -1.0, q64, 0.0, nullptr, nullptr, r64);
        CK(cudaGetLastError(), "k_lin launch");
        return twin_wnorm(H, X, r64, &rr2, st);
    };
    if ((rc = true_residual())) return rc;
    double rel = bn2 > 0.0 ? std::sqrt(std::max(rr2, 0.0) / bn2) : 0.0;
    int done = 0;
    if (bn2 > 0.0 && rr2 > 0.0 && rel > tol && max_iters > 0) {
        double sc = std::sqrt(rr2);
        VecArgs<float> v = vec_args<float>(H, x32, 0);
        CK(cudaMemsetAsync(x32, 0, n * sizeof(float), st), "solve increment");
        k_refresh<float><<<H->npart, PBLK, 0, st>>>(n, r64, 1.0 / sc, 0.0, 1, 0.0, v);
        CK(cudaGetLastError(), "k_refresh launch");
        double rz[2] = {0.0, 0.0};
        CK(cudaMemcpyAsync(rz, H->rztot, sizeof(double), cudaMemcpyDeviceToHost, st), "solve rz");
        CK(cudaStreamSynchronize(st), "solve rz");
        double rz_upd = rz[0];
        int j0 = 0;
        for (;;) {
            const int k = std::min(FEWHA_MAX_ITERS - j0, max_iters - done);
            for (int j = j0; j < j0 + k; ++j) {
                if ((rc = enqueue_apply<float>(H, d, p, q, j, j > 0, st))) return rc;
                if ((rc = launch_vec<float, V_UPDATE>(H, n, vec_args<float>(H, x32, j), st))) return rc;
            }
            done += k;
            const int last = j0 + k;
            CK(cudaMemcpyAsync(rz, H->rztot + last - 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, st),
               "solve rz");
            CK(cudaStreamSynchronize(st), "solve rz");
            const bool stopped = !(rz[1] > 0.0) || !std::isfinite(rz[1]);
            const bool fold = stopped || done >= max_iters || rz[1] < DELTA * DELTA * rz_upd ||
                              sc * std::sqrt(rz[1]) <= tol * std::sqrt(bn2);
            if (!fold) {
                // continue the recurrence: slots (last - 1, last) -> (0, 1)
                CK(cudaMemcpyAsync(H->rztot, H->rztot + last - 1, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st),
                   "solve resume");
                j0 = 1;
                continue;
            }
            k_accum<float><<<gl, PBLK, 0, st>>>(n, sc, x32, x64);
            CK(cudaGetLastError(), "k_accum launch");
            if ((rc = true_residual())) return rc;
            rel = std::sqrt(std::max(rr2, 0.0) / bn2);
            if (!std::isfinite(rr2)) break;
            if (rel <= tol || done >= max_iters || !(rr2 > 0.0) || stopped) break;
            const double scn = std::sqrt(rr2), ratio = sc / scn;
            k_refresh<float><<<H->npart, PBLK, 0, st>>>(n, r64, 1.0 / scn, ratio, 0, rz[0] * ratio * ratio, v);
            CK(cudaGetLastError(), "k_refresh launch");
            CK(cudaMemcpyAsync(&rz_upd, H->rztot + 1, sizeof(double), cudaMemcpyDeviceToHost, st), "solve rz");
            CK(cudaStreamSynchronize(st), "solve rz");
            sc = scn;
            j0 = 1;
        }
    }
    H->have_prev = false;
    if (iters_out) *iters_out = done;
    if (rel_out) *rel_out = rel;
    if (!std::isfinite(rr2)) return fail(H, FEWHA_ERR_NONFINITE, "non-finite residual in the converged solve");
    return FEWHA_OK;
}

template <class T>
int reconstruct_converged(fewha_handle* H, const T* s, T* dm, double tol, int max_iters, int* iters,
                          double* rel, cudaStream_t st) {
    const Desc<T> d = make_desc<T>(H);
    int rc;
    H->grad_ready = false;
    if constexpr (sizeof(T) == 4) {
        // single precision: the rhs, the iterate c* and the fit in double on the twin, the
        // solve's iterations in float (reliable_solve)
        if ((rc = ensure_twin(H))) return rc;
        fewha_handle* X = H->twin;
        const Desc<double> dx = make_desc<double>(X);
        double* s64 = static_cast<double*>(X->s_tmp);
        k_convert<double, float><<<(d.n_s + 255) / 256, 256, 0, st>>>(d.n_s, s, s64);
        CK(cudaGetLastError(), "k_convert launch");
        if ((rc = enqueue_rhs<double>(X, dx, s64, static_cast<double*>(X->b), st))) return fail(H, rc, X->err);
        if ((rc = reliable_solve(H, X, static_cast<const double*>(X->b), static_cast<double*>(X->cgrad),
                                 X->have_cgrad, tol, max_iters, st, iters, rel)))
            return rc;
        X->have_cgrad = true;
        double* dm64 = static_cast<double*>(X->dm_tmp);
        if ((rc = enqueue_fit<double>(X, dx, static_cast<const double*>(X->cgrad), dm64, false, st)))
            return fail(H, rc, X->err);
        k_convert<float, double><<<(d.n_act + 255) / 256, 256, 0, st>>>(d.n_act, dm64, dm);
        CK(cudaGetLastError(), "k_convert launch");
    } else {
        if ((rc = enqueue_rhs<T>(H, d, s, static_cast<T*>(H->b), st))) return rc;
        // warm start from the previous converged solution (a nearby M or b)
        if ((rc = solve_converged<T>(H, static_cast<const T*>(H->b), static_cast<T*>(H->cgrad), H->have_cgrad, tol,
                                     max_iters, st, iters, rel)))
            return rc;
        H->have_cgrad = true;
        if ((rc = enqueue_fit<T>(H, d, static_cast<const T*>(H->cgrad), dm, false, st))) return rc;
    }
    H->grad_ready = true;
    H->grad_tol = tol;
    H->grad_max_iters = max_iters;
    return FEWHA_OK;
}

// Gradients of J(a~) at the last converged reconstruction, given g_a = dJ/da~:
//   lambda = M^-1 (F W^T)^T g_a,  dJ/ds = C_hat^-1 Gamma P W^T lambda,
//   dJ/dalpha = -lambda^T D c*,   dJ/dw_l = alpha lambda_l^T D_l c*_l / w_l.
// The single-precision form solves for lambda with reliable_solve and forms every other
// step (F^T, the slope map, the per-layer sums) in double on the twin.
template <class T>
int backward(fewha_handle* H, const T* g_a, T* g_s, double* g_alpha, double* g_w, cudaStream_t st) {
    if (!H->grad_ready) return fail(H, FEWHA_ERR_INVALID_ARG, "no converged reconstruction to differentiate");
    const Desc<T> d = make_desc<T>(H);
    int rc;
    int it = 0;
    double rel = 0.0;
    double S[MAXL];
    if constexpr (sizeof(T) == 4) {
        fewha_handle* X = H->twin;
        const Desc<double> dx = make_desc<double>(X);
        double* ga64 = static_cast<double*>(X->dm_tmp);
        double* b64 = static_cast<double*>(X->b);
        double* lam = static_cast<double*>(X->lam);
        k_convert<double, float><<<(d.n_act + 255) / 256, 256, 0, st>>>(d.n_act, g_a, ga64);
        CK(cudaGetLastError(), "k_convert launch");
        if ((rc = launch_layer<double, LSRC_DM, LDST_COEF, false>(X, dx, layer_args<double>(X, ga64, b64), st)))
            return fail(H, rc, X->err);
        if ((rc = reliable_solve(H, X, b64, lam, X->have_lam, H->grad_tol, H->grad_max_iters, st, &it, &rel)))
            return rc;
        X->have_lam = true;
        if (g_s) {
            double* lz = static_cast<double*>(X->c_tmp);
            double* phi = static_cast<double*>(X->phi);
            double* t1 = static_cast<double*>(X->s_tmp);
            double* t2 = static_cast<double*>(X->s_pol);
            CK(cudaMemcpyAsync(lz, lam, d.n_c * sizeof(double), cudaMemcpyDeviceToDevice, st), "lambda copy");
            if ((rc = zero_pistons<double>(H, lz, st))) return rc;
            if ((rc = launch_layer<double, LSRC_COEF, LDST_PHI, false>(X, dx, layer_args<double>(X, lz, phi), st)) ||
                (rc = launch_sensor<double, SSRC_PHI, false, SDST_SLOPES>(X, dx, phi, t1, st)) ||
                (rc = launch_sensor<double, SSRC_SLOPES, true, SDST_SLOPES>(X, dx, t1, t2, st)))
                return fail(H, rc, X->err);
            k_convert<float, double><<<(d.n_s + 255) / 256, 256, 0, st>>>(d.n_s, t2, g_s);
            CK(cudaGetLastError(), "k_convert launch");
        }
        k_layer_dots<double><<<d.n_layers, PBLK, 0, st>>>(dx, lam, static_cast<const double*>(X->cgrad), X->gdot);
        CK(cudaGetLastError(), "k_layer_dots launch");
        CK(cudaMemcpyAsync(S, X->gdot, d.n_layers * sizeof(double), cudaMemcpyDeviceToHost, st), "layer sums");
    } else {
        T* b = static_cast<T*>(H->b);
        T* lam = static_cast<T*>(H->lam);
        T* phi = static_cast<T*>(H->phi);
        T* st_s = static_cast<T*>(H->s_tmp);
        if ((rc = launch_layer<T, LSRC_DM, LDST_COEF, false>(H, d, layer_args<T>(H, g_a, b), st))) return rc;
        if ((rc = solve_converged<T>(H, b, lam, H->have_lam, H->grad_tol, H->grad_max_iters, st, &it, &rel)))
            return rc;
        H->have_lam = true;
        if (g_s) {
            T* lz = static_cast<T*>(H->c_tmp);
            CK(cudaMemcpyAsync(lz, lam, d.n_c * sizeof(T), cudaMemcpyDeviceToDevice, st), "lambda copy");
            if ((rc = zero_pistons<T>(H, lz, st))) return rc;
            if ((rc = launch_layer<T, LSRC_COEF, LDST_PHI, false>(H, d, layer_args<T>(H, lz, phi), st))) return rc;
            if ((rc = launch_sensor<T, SSRC_PHI, false, SDST_SLOPES>(H, d, phi, st_s, st))) return rc;
            if ((rc = launch_sensor<T, SSRC_SLOPES, true, SDST_SLOPES>(H, d, st_s, g_s, st))) return rc;
        }
        k_layer_dots<T><<<d.n_layers, PBLK, 0, st>>>(d, lam, static_cast<const T*>(H->cgrad), H->gdot);
        CK(cudaGetLastError(), "k_layer_dots launch");
        CK(cudaMemcpyAsync(S, H->gdot, d.n_layers * sizeof(double), cudaMemcpyDeviceToHost, st), "layer sums");
    }
    CK(cudaStreamSynchronize(st), "backward");
    double tot = 0.0;
    for (int l = 0; l < d.n_layers; ++l) tot += S[l];
    if (g_alpha) *g_alpha = -tot;
    if (g_w)
        for (int l = 0; l < d.n_layers; ++l) g_w[l] = H->params.alpha * S[l] / H->weights[l];
    return FEWHA_OK;
}

// x = M^-1 b from x = 0 (fewha_solve): the double-precision form by solve_converged, the
// single-precision form by reliable_solve with b and x converted at the ends.
template <class T>
int solve_entry(fewha_handle* H, const T* b, T* x, double tol, int max_iters, cudaStream_t st, int* iters,
                double* rel) {
    if constexpr (sizeof(T) == 4) {
        int rc;
        if ((rc = ensure_twin(H))) return rc;
        fewha_handle* X = H->twin;
        const int n = H->setup.n_c;
        double* b64 = static_cast<double*>(X->b);
        double* x64 = static_cast<double*>(X->c_tmp);
        k_convert<double, float><<<(n + 255) / 256, 256, 0, st>>>(n, b, b64);
        CK(cudaGetLastError(), "k_convert launch");
        if ((rc = reliable_solve(H, X, b64, x64, false, tol, max_iters, st, iters, rel))) return rc;
        k_convert<float, double><<<(n + 255) / 256, 256, 0, st>>>(n, x64, x);
        CK(cudaGetLastError(), "k_convert launch");
        CK(cudaStreamSynchronize(st), "solve");
        return FEWHA_OK;
    } else {
        return solve_converged<T>(H, b, x, false, tol, max_iters, st, iters, rel);
    }
}

// Reverse mode through the fixed-iteration frame: the forward recurrence from c0 with
// every vector kept, then each statement's adjoint in reverse order (M and J^-1 are
// symmetric), three vector kernels and one M-apply per iteration (k_vjp).  The scalars
// (rho, sigma, alpha, beta and their adjoints) stay on the device; the host synchronises
// once, at the end.  Synchronous.
// ---- least-squares fit over fitting directions (Sec. 4.1) --------------------------

int check_lsfit(fewha_handle* H, const fewha_lsfit* cfg) {
    if (!cfg || !cfg->theta_x || !cfg->theta_y || !cfg->weight)
        return fail(H, FEWHA_ERR_INVALID_ARG, "fit_ls: null configuration or direction array");
    if (cfg->n_dirs < 1 || cfg->n_dirs > FEWHA_MAX_FIT_DIRS)
        return fail(H, FEWHA_ERR_INVALID_ARG, "fit_ls: n_dirs out of 1 .. FEWHA_MAX_FIT_DIRS");
    if (cfg->n_fit < 1 || cfg->n_fit > FEWHA_MAX_FIT_NODES)
        return fail(H, FEWHA_ERR_INVALID_ARG, "fit_ls: n_fit out of 1 .. FEWHA_MAX_FIT_NODES");
    if (!(cfg->eps >= 0.0) || !std::isfinite(cfg->eps))
        return fail(H, FEWHA_ERR_INVALID_ARG, "fit_ls: eps must be finite and >= 0");
    bool any = false;
    for (int k = 0; k < cfg->n_dirs; ++k) {
        if (!std::isfinite(cfg->theta_x[k]) || !std::isfinite(cfg->theta_y[k]) || !(cfg->weight[k] >= 0.0) ||
            !std::isfinite(cfg->weight[k]))
            return fail(H, FEWHA_ERR_INVALID_ARG, "fit_ls: directions must be finite and weights finite and >= 0");
        any = any || cfg->weight[k] > 0.0;
    }
    if (!any) return fail(H, FEWHA_ERR_INVALID_ARG, "fit_ls: no positive weight");
    return FEWHA_OK;
}

// Grow a group of device buffers to `need` elements each (new buffers when the group's
// capacity *cap is smaller; the old ones stay on the handle's list until it is destroyed).
template <class X>
int lsf_grow(fewha_handle* H, std::initializer_list<X**> ptrs, size_t* cap, size_t need) {
    if (*cap >= need) return FEWHA_OK;
    for (X** p : ptrs) {
        int rc = dalloc(H, p, need);
        if (rc) return rc;
    }
    *cap = need;
    return FEWHA_OK;
}

int lsf_grow_t(fewha_handle* H, std::initializer_list<void**> ptrs, size_t* cap, size_t need) {
    if (*cap >= need) return FEWHA_OK;
    for (void** p : ptrs) {
        int rc = talloc(H, p, need);
        if (rc) return rc;
    }
    *cap = need;
    return FEWHA_OK;
}

template <class T>
int lsf_upload(fewha_handle* H, void* dst, const std::vector<double>& src) {
    std::vector<T> t(src.begin(), src.end());
    return upload(H, static_cast<T*>(dst), t);
}

// Tables of configuration `cfg` on the device (built unless they already are).
template <class T>
int ensure_lsfit(fewha_handle* H, const fewha_lsfit& cfg) {
    std::vector<double> key{double(cfg.n_dirs), double(cfg.n_fit), cfg.eps};
    for (int k = 0; k < cfg.n_dirs; ++k) {
        key.push_back(cfg.theta_x[k]);
        key.push_back(cfg.theta_y[k]);
        key.push_back(cfg.weight[k]);
    }
    if (!H->lsf) H->lsf = new LsfitDev();
    LsfitDev& F = *H->lsf;
    if (F.key == key) return FEWHA_OK;
    F.key.clear();
    std::string err;
    int rc = build_lsfit(H->setup, H->tel_in.obs, H->dms_in.data(), cfg, F.host, err);
    if (rc) return fail(H, rc, "fit_ls: " + err);
    const LsfitHost& L = F.host;
    const size_t n_a = static_cast<size_t>(H->setup.n_act);
    const size_t nb = (n_a + LSF_ABLK - 1) / LSF_ABLK;
    if (!F.state) {   // allocated last: all of them are there
        if ((rc = talloc(H, &F.r, n_a)) || (rc = talloc(H, &F.p, n_a)) || (rc = talloc(H, &F.q, n_a)) ||
            (rc = dalloc(H, &F.part, nb)) || (rc = dalloc(H, &F.msum, LSF_MAXSL)) || (rc = dalloc(H, &F.sc, 2)) ||
            (rc = dalloc(H, &F.state, 2)))
            return rc;
    }
    if ((rc = lsf_grow<unsigned char>(H, {&F.mask}, &F.cap_pix, L.mask.size())) ||
        (rc = lsf_grow<int>(H, {&F.ly0, &F.lx0}, &F.cap_l, L.ly0.size())) ||
        (rc = lsf_grow_t(H, {&F.lfy, &F.lfx}, &F.cap_lf, L.lfy.size())) ||
        (rc = lsf_grow<int>(H, {&F.my0, &F.mx0}, &F.cap_m, L.my0.size())) ||
        (rc = lsf_grow_t(H, {&F.mfy, &F.mfx}, &F.cap_mf, L.mfy.size())) ||
        (rc = lsf_grow<int>(H, {&F.ylo, &F.yhi, &F.xlo, &F.xhi}, &F.cap_rng, L.ylo.size())) ||
        (rc = lsf_grow_t(H, {&F.v}, &F.cap_v, static_cast<size_t>(L.n_dirs) * L.mask.size())))
        return rc;
    if ((rc = upload(H, F.mask, L.mask)) || (rc = upload(H, F.ly0, L.ly0)) || (rc = upload(H, F.lx0, L.lx0)) ||
        (rc = lsf_upload<T>(H, F.lfy, L.lfy)) || (rc = lsf_upload<T>(H, F.lfx, L.lfx)) ||
        (rc = upload(H, F.my0, L.my0)) || (rc = upload(H, F.mx0, L.mx0)) ||
        (rc = lsf_upload<T>(H, F.mfy, L.mfy)) || (rc = lsf_upload<T>(H, F.mfx, L.mfx)) ||
        (rc = upload(H, F.ylo, L.ylo)) || (rc = upload(H, F.yhi, L.yhi)) || (rc = upload(H, F.xlo, L.xlo)) ||
        (rc = upload(H, F.xhi, L.xhi)))
        return rc;
    F.key = key;
    return FEWHA_OK;
}

template <class T>
LsDesc<T> lsf_desc(const fewha_handle* H, const fewha_lsfit& cfg) {
    const LsfitDev& F = *H->lsf;
    const HostSetup& S = H->setup;
    LsDesc<T> d{};
    d.n_dirs = F.host.n_dirs;
    d.nf1 = F.host.nf1;
    d.n_pup = F.host.n_pup;
    // slices of each direction's pupil grid: about one node per thread, at most LSF_MAXSL
    // (direction, slice) CTAs in all
    d.n_slices = std::max(1, std::min((d.nf1 * d.nf1 + LSF_SBLK - 1) / LSF_SBLK, LSF_MAXSL / d.n_dirs));
    d.n_layers = static_cast<int>(S.L.size());
    d.n_dms = static_cast<int>(S.Mi.size());
    d.n_a = S.n_act;
    for (int l = 0; l < d.n_layers; ++l) {
        d.lay_n[l] = S.L[l].n;
        d.lay_off[l] = S.L[l].off;
    }
    for (int m = 0; m < d.n_dms; ++m) {
        d.dm_n[m] = S.Mi[m].n_act;
        d.dm_off[m] = S.Mi[m].off;
    }
    for (int k = 0; k < d.n_dirs; ++k) d.w[k] = static_cast<T>(cfg.weight[k]);
    d.eps = static_cast<T>(cfg.eps);
    d.mask = F.mask;
    d.ly0 = F.ly0;
    d.lx0 = F.lx0;
    d.my0 = F.my0;
    d.mx0 = F.mx0;
    d.lfy = static_cast<const T*>(F.lfy);
    d.lfx = static_cast<const T*>(F.lfx);
    d.mfy = static_cast<const T*>(F.mfy);
    d.mfx = static_cast<const T*>(F.mfx);
    d.ylo = F.ylo;
    d.yhi = F.yhi;
    d.xlo = F.xlo;
    d.xhi = F.xhi;
    return d;
}

// phi = W^T c, the right-hand side, then CG chunks of FEWHA_MAX_ITERS steps until the
// device reports that the CG has stopped.
template <class T>
int fit_ls(fewha_handle* H, const fewha_lsfit& cfg, const T* c, T* a, double tol, int max_iters, int* iters_out,
           double* rel_out, cudaStream_t st) {
    int rc = ensure_lsfit<T>(H, cfg);
    if (rc) return rc;
    LsfitDev& F = *H->lsf;
    const Desc<T> d = make_desc<T>(H);
    T* phi = static_cast<T*>(H->phi);
    if ((rc = launch_layer<T, LSRC_COEF, LDST_PHI, false>(H, d, layer_args<T>(H, c, phi), st))) return rc;
    const LsDesc<T> ld = lsf_desc<T>(H, cfg);
    T* v = static_cast<T*>(F.v);
    T* p = static_cast<T*>(F.p);
    T* q = static_cast<T*>(F.q);
    const int nb = (ld.n_a + LSF_ABLK - 1) / LSF_ABLK;
    const dim3 sgrid(ld.n_slices, ld.n_dirs);
    k_lsf_sample<T, true><<<sgrid, LSF_SBLK, 0, st>>>(ld, phi, v, F.msum, nullptr);
    k_lsf_adj<T><<<nb, LSF_ABLK, 0, st>>>(ld, v, F.msum, nullptr, q, nullptr, nullptr);
    LsCg<T> g{};
    g.n = ld.n_a;
    g.nparts = nb;
    g.max_iters = max_iters;
    g.tol2 = tol * tol;
    g.a = a;
    g.r = static_cast<T*>(F.r);
    g.p = p;
    g.q = q;
    g.part = F.part;
    g.sc = F.sc;
    g.state = F.state;
    k_lsf_cg<T, true><<<1, LSF_CBLK, 0, st>>>(g);
    CK(cudaGetLastError(), "fit_ls launch");
    int hst[2] = {0, 0};
    double hsc[2] = {0.0, 0.0};
    int run = 0;
    for (;;) {
        const int k = std::min(FEWHA_MAX_ITERS, max_iters - run);
        for (int j = 0; j < k; ++j) {
            k_lsf_sample<T, false><<<sgrid, LSF_SBLK, 0, st>>>(ld, p, v, F.msum, F.state);
            k_lsf_adj<T><<<nb, LSF_ABLK, 0, st>>>(ld, v, F.msum, p, q, F.part, F.state);
            k_lsf_cg<T, false><<<1, LSF_CBLK, 0, st>>>(g);
        }
        CK(cudaGetLastError(), "fit_ls launch");
        run += k;
        CK(cudaMemcpyAsync(hst, F.state, sizeof hst, cudaMemcpyDeviceToHost, st), "fit_ls state");
        CK(cudaMemcpyAsync(hsc, F.sc, sizeof hsc, cudaMemcpyDeviceToHost, st), "fit_ls state");
        CK(cudaStreamSynchronize(st), "fit_ls");
        if (hst[0] || run >= max_iters) break;
    }
    if (iters_out) *iters_out = hst[1];
    if (rel_out) *rel_out = hsc[1] > 0.0 ? std::sqrt(std::max(hsc[0], 0.0) / hsc[1]) : 0.0;
    if (!std::isfinite(hsc[0]) || !std::isfinite(hsc[1]))
        return fail(H, FEWHA_ERR_NONFINITE, "fit_ls: non-finite residual");
    if (hst[0] == 2) return fail(H, FEWHA_ERR_NONFINITE, "fit_ls: CG breakdown (p.q <= 0)");
    return FEWHA_OK;
}

template <class T>
int frame_vjp(fewha_handle* H, const T* s, const T* c0, const T* g_a, T* dm, T* g_s, cudaStream_t st) {
    const Desc<T> d = make_desc<T>(H);
    const int k = H->params.iters, n = d.n_c;
    const size_t ld = (static_cast<size_t>(n) + 63) & ~static_cast<size_t>(63);
    const size_t need = (4 * static_cast<size_t>(k + 1) + 8) * ld;
    if (H->vjp_cap < need) {
        if (H->vjp) {
            cudaFree(H->vjp);
            const size_t at = std::find(H->allocs.begin(), H->allocs.end(), H->vjp) - H->allocs.begin();
            H->allocs.erase(H->allocs.begin() + at);
            H->alloc_sizes.erase(H->alloc_sizes.begin() + at);
            H->vjp = nullptr;
        }
        int rc0;
        if ((rc0 = talloc(H, &H->vjp, need))) return rc0;
        H->vjp_cap = need;
    }
    T* base = static_cast<T*>(H->vjp);
    T* R = base;                                   // r_0 .. r_k
    T* Z = R + (k + 1) * ld;                       // z_0 .. z_k
    T* P = Z + (k + 1) * ld;                       // p_0 .. p_(k-1) (p_k unused)
    T* Q = P + (k + 1) * ld;                       // q_0 .. q_(k-1)
    T* c = Q + (k + 1) * ld;
    T* scratch = c + ld;
    T* cbar = scratch + ld;
    T* rbar = cbar + ld;
    T* pbar = rbar + ld;
    T* pbi = pbar + ld;
    T* qbar = pbi + ld;
    const T* Jinv = static_cast<const T*>(H->Jinv);
    int rc;
    // ---- forward: b, r0 = b - M c0, then the iterations, every vector kept -------------
    if ((rc = enqueue_rhs<T>(H, d, s, static_cast<T*>(H->b), st))) return rc;
    CK(cudaMemcpyAsync(c, c0, n * sizeof(T), cudaMemcpyDeviceToDevice, st), "vjp c0");
    if ((rc = enqueue_apply<T>(H, d, c, static_cast<T*>(H->q), PQ_SCRATCH_SLOT, false, st))) return rc;
    VecArgs<T> v = vec_args<T>(H, c, 0);
    v.r = R;
    v.z = Z;
    v.p = P;
    v.b_prev = scratch;                            // the handle's b_prev stays untouched
    if ((rc = launch_vec<T, V_INIT>(H, n, v, st))) return rc;
    AugArgs<T> a{};
    a.m = 0;
    for (int i = 0; i < k; ++i) {
        // p_i = z_i + beta p_(i-1) into its own slot, fused into the apply's inverse kernel
        if (i > 0)
            rc = enqueue_apply_aug<T>(H, d, P + (i - 1) * ld, P + i * ld, Z + i * ld, Q + i * ld, i, a, st);
        else
            rc = enqueue_apply<T>(H, d, P, Q, 0, false, st);
        if (rc) return rc;
        CK(cudaMemcpyAsync(R + (i + 1) * ld, R + i * ld, n * sizeof(T), cudaMemcpyDeviceToDevice, st), "vjp r");
        VecArgs<T> w = vec_args<T>(H, c, i);
        w.p = P + i * ld;
        w.q = Q + i * ld;
        w.r = R + (i + 1) * ld;
        w.z = Z + (i + 1) * ld;
        if ((rc = launch_vec<T, V_UPDATE>(H, n, w, st))) return rc;
    }
    if (dm && (rc = enqueue_fit<T>(H, d, c, dm, false, st))) return rc;
    if (!g_a) {
        CK(cudaStreamSynchronize(st), "vjp forward");
        return FEWHA_OK;
    }
    // ---- reverse: every scalar on the device, no host round trip until the end ----------
    if ((rc = launch_layer<T, LSRC_DM, LDST_COEF, false>(H, d, layer_args<T>(H, g_a, cbar), st))) return rc;
    CK(cudaMemsetAsync(rbar, 0, n * sizeof(T), st), "vjp zero");
    CK(cudaMemsetAsync(pbar, 0, n * sizeof(T), st), "vjp zero");
    CK(cudaMemsetAsync(H->gdot, 0, 4 * sizeof(double), st), "vjp scalars");
    VjpArgs<T> va;
    va.rbar = rbar;
    va.pbar = pbar;
    va.pbi = pbi;
    va.qbar = qbar;
    va.cbar = cbar;
    va.Mq = scratch;
    va.Jinv = Jinv;
    va.rho = H->rztot;
    va.sigma = H->pqtot;
    va.rs = H->gdot;
    va.part = H->rzpart + static_cast<size_t>(FEWHA_MAX_ITERS + 1) * NPART_MAX;   // a free slot pair
    va.count = H->count;
    va.npart = NPART_MAX / 2;
    const int gv = std::min(NPART_MAX / 2, (n + PBLK - 1) / PBLK);
    for (int i = k - 1; i >= 0; --i) {
        va.i = i;
        va.first = i == k - 1;
        va.p = P + i * ld;
        va.q = Q + i * ld;
        va.r1 = R + (i + 1) * ld;
        va.z1 = Z + (i + 1) * ld;
        k_vjp<T, VJ_A><<<gv, PBLK, 0, st>>>(n, va);
        k_vjp<T, VJ_B><<<gv, PBLK, 0, st>>>(n, va);
        k_vjp<T, VJ_C><<<gv, PBLK, 0, st>>>(n, va);
        CK(cudaGetLastError(), "k_vjp launch");
        // q_i = M p_i: p_bar_i += M q_bar (added by the next VJ_A, or VJ_E)
        if ((rc = enqueue_apply<T>(H, d, qbar, scratch, PQ_SCRATCH_SLOT, false, st))) return rc;
    }
    // p_0 = z_0, rho_0 = r_0 . z_0, z_0 = J^-1 r_0, r_0 = b - M c0: b_bar = r_bar_0
    if (k > 0) {
        va.r1 = R;
        va.z1 = Z;
        k_vjp<T, VJ_E><<<gv, PBLK, 0, st>>>(n, va);
        CK(cudaGetLastError(), "k_vjp launch");
    }
    // the recurrence must not have stopped (r.z or p.q vanished): checked once, at the end
    std::vector<double> rho(k + 1), sigma(k + 1);
    CK(cudaMemcpyAsync(rho.data(), H->rztot, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, st), "vjp rho");
    if (k > 0)
        CK(cudaMemcpyAsync(sigma.data(), H->pqtot, k * sizeof(double), cudaMemcpyDeviceToHost, st), "vjp sigma");
    // dJ/ds = C_hat^-1 Gamma P W^T b_bar (b_bar's pistons, large and annihilated by Gamma,
    // left out first)
    T* phi = static_cast<T*>(H->phi);
    T* st_s = static_cast<T*>(H->s_tmp);
    if ((rc = zero_pistons<T>(H, rbar, st))) return rc;
    if ((rc = launch_layer<T, LSRC_COEF, LDST_PHI, false>(H, d, layer_args<T>(H, rbar, phi), st))) return rc;
    if ((rc = launch_sensor<T, SSRC_PHI, false, SDST_SLOPES>(H, d, phi, st_s, st))) return rc;
    if ((rc = launch_sensor<T, SSRC_SLOPES, true, SDST_SLOPES>(H, d, st_s, g_s, st))) return rc;
    CK(cudaStreamSynchronize(st), "vjp");
    for (int i = 0; i < k; ++i)
        if (!(sigma[i] > 0.0) || rho[i] == 0.0)
            return fail(H, FEWHA_ERR_NONFINITE, "the frame's recurrence stopped (r.z or p.q vanished)");
    return FEWHA_OK;
}

// ---------------------------------------------------------------- batched frames
int bfail(fewha_batch* B, int code, const std::string& msg) {
    if (B) B->err = msg;
    return code;
}

#define BCK(call, where)                                                                      \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return bfail(B, FEWHA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

size_t round16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

template <class T>
size_t barg_size(int kind) {
    switch (kind) {
        case BK_INV: case BK_INV_UPD: case BK_FWD_APPLY: case BK_FWD_COEF: case BK_FWD_RINIT:
            return sizeof(ClArgs<T>);
        case BK_SEN_PHI: case BK_SEN_SLOPES: case BK_SEN_RESID: return sizeof(SensorArgs<T>);
        case BK_PROJ: case BK_PROJT: return sizeof(const T*);
        case BK_FIT: return sizeof(FitArgs<T>);
        default: return sizeof(VecArgs<T>);
    }
}

size_t bsmem(const fewha_handle* H, int kind) {
    switch (kind) {
        case BK_INV: case BK_INV_UPD: return H->smem_inv;
        case BK_FWD_APPLY: case BK_FWD_COEF: case BK_FWD_RINIT: return H->smem_fwd;
        case BK_SEN_PHI: case BK_SEN_SLOPES: case BK_SEN_RESID: return H->smem_sen;
        case BK_PROJ: return H->smem_proj;
        case BK_PROJT: return H->smem_projT;
        default: return 0;
    }
}

// Relative work of one instance's frame: the wavelet transforms scale with n_c, the
// projections with layers x aperture nodes.
double bcost(const fewha_handle* H) {
    return 2.0 * H->setup.n_c + static_cast<double>(H->setup.L.size()) * H->setup.n_nodes;
}

int bnparts(const fewha_handle* H, int vec_passes, int vec_threads) {
    const int per = (vec_threads ? vec_threads : PBLK) * PVEC * vec_passes;
    int n = (H->setup.n_c + per - 1) / per;
    return n < 1 ? 1 : (n > NPART_MAX ? NPART_MAX : n);
}

// Record every member's frame (host only) and check that the step sequences agree.
template <class T>
int batch_record(fewha_batch* B, const T* const* s, T* const* dm, bool warm, std::vector<Recorder<T>>& recs) {
    const size_t n = B->h.size();
    recs.assign(n, Recorder<T>());
    for (size_t i = 0; i < n; ++i) {
        fewha_handle* H = B->h[i];
        if (!s[i] || !dm[i]) return bfail(B, FEWHA_ERR_INVALID_ARG, "null slope or DM pointer of instance " + std::to_string(i));
        if (H->params.flags & FEWHA_FLAG_AUGMENTED)
            return bfail(B, FEWHA_ERR_INVALID_ARG, "augmented PCG frames are not batched (instance " + std::to_string(i) + ")");
        if (H->params.flags & FEWHA_FLAG_CLOSED_LOOP)
            return bfail(B, FEWHA_ERR_INVALID_ARG, "closed-loop frames are not batched (instance " + std::to_string(i) + ")");
        g_recorder = &recs[i];
        const int rc = enqueue_frame<T>(H, s[i], static_cast<T*>(H->c), dm[i], warm, nullptr);
        g_recorder = nullptr;
        if (rc) return bfail(B, rc, "instance " + std::to_string(i) + ": " + H->err);
        bool same = recs[i].steps.size() == recs[0].steps.size();
        for (size_t j = 0; same && j < recs[i].steps.size(); ++j) same = recs[i].steps[j].kind == recs[0].steps[j].kind;
        if (!same) return bfail(B, FEWHA_ERR_INVALID_ARG, "instances differ in iteration count or residual mode");
    }
    return FEWHA_OK;
}

// Argument table: per step, one entry per instance, each step's array 16-byte aligned.
template <class T>
void batch_pack(const std::vector<Recorder<T>>& recs, const std::vector<int>& nparts,
                std::vector<unsigned char>& out, std::vector<size_t>& offs) {
    const size_t n = recs.size(), S = recs[0].steps.size();
    offs.assign(S, 0);
    size_t off = 0;
    for (size_t j = 0; j < S; ++j) {
        offs[j] = off;
        off += round16(n * barg_size<T>(recs[0].steps[j].kind));
    }
    out.assign(off, 0);
    for (size_t j = 0; j < S; ++j) {
        const int kind = recs[0].steps[j].kind;
        const size_t sz = barg_size<T>(kind);
        for (size_t i = 0; i < n; ++i) {
            const BStep<T>& st = recs[i].steps[j];
            unsigned char* dst = out.data() + offs[j] + i * sz;
            switch (bkind_list(kind)) {
                case BL_LAYER: std::memcpy(dst, &st.cl, sz); break;
                case BL_SENSOR: std::memcpy(dst, &st.sa, sz); break;
                case BL_PAIR: std::memcpy(dst, &st.ptr, sz); break;
                case BL_FIT: std::memcpy(dst, &st.fa, sz); break;
                default: {
                    VecArgs<T> v = st.va;
                    v.pcg.npart = nparts[i];
                    std::memcpy(dst, &v, sz);
                }
            }
        }
    }
}

void batch_drop_plan(fewha_batch* B) {
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
    if (B->dev) cudaFree(B->dev);
    B->dev = nullptr;
    B->have_plan = false;
}

// Build the device block and capture the graph of one batched frame.
template <class T>
int batch_build(fewha_batch* B, const std::vector<Recorder<T>>& recs, const std::vector<int>& nparts,
                const std::vector<unsigned char>& args, const std::vector<size_t>& offs, bool warm) {
    const int n = static_cast<int>(B->h.size());
    const fewha_batch_config cfg = B->cfg;
    BCK(cudaDeviceSynchronize(), "batch sync");
    batch_drop_plan(B);
    // order and groups (greedy balanced partition by cost, costliest first)
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) cost[i] = bcost(B->h[i]);
    std::vector<int> byc(n);
    for (int i = 0; i < n; ++i) byc[i] = i;
    std::stable_sort(byc.begin(), byc.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    const int G = std::max(1, std::min(cfg.groups, n));
    std::vector<int> grp(n, 0);
    std::vector<double> load(G, 0.0);
    for (int i : byc) {
        const int g = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
        grp[i] = g;
        load[g] += cost[i];
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = cfg.order == 1 ? byc[i] : i;
    // work lists per group
    std::vector<std::vector<BItem>> lists(G * BL_COUNT);
    for (int i : order) {
        const fewha_handle* H = B->h[i];
        const int g = grp[i], nl = static_cast<int>(H->setup.L.size()), nw = static_cast<int>(H->setup.G.size());
        for (int l = 0; l < nl; ++l) lists[g * BL_COUNT + BL_LAYER].push_back({i, l});
        for (int w = 0; w < nw; ++w) lists[g * BL_COUNT + BL_SENSOR].push_back({i, w});
        for (int w = 0; w < nw; ++w)
            for (int l = 0; l < nl; ++l) lists[g * BL_COUNT + BL_PAIR].push_back({i, w * MAXL + l});
        for (int k = 0; k < nparts[i]; ++k) lists[g * BL_COUNT + BL_VEC].push_back({i, k});
        for (int k = 0; k < (H->setup.n_act + PBLK - 1) / PBLK; ++k) lists[g * BL_COUNT + BL_FIT].push_back({i, k});
    }
    // instances
    std::vector<BInst<T>> inst(n);
    for (int i = 0; i < n; ++i) {
        fewha_handle* H = B->h[i];
        BInst<T>& I = inst[i];
        std::memset(&I, 0, sizeof(I));
        I.d = make_desc<T>(H);
        I.lay_fwd = H->lay_fwd;
        I.lay_inv = H->lay_inv;
        I.lay_sen = H->lay_sen;
        I.pb = pair_bufs<T>(H);
        I.desc_bytes = static_cast<int>(offsetof(Desc<T>, box) + static_cast<size_t>(I.d.n_wfs) * MAXL * 4 * sizeof(int));
        I.ctas_layer = static_cast<unsigned>(CL * I.d.n_layers);
        I.nparts = nparts[i];
    }
    // device block
    const size_t inst_bytes = round16(sizeof(BInst<T>) * n);
    std::vector<size_t> loff(lists.size());
    size_t off = inst_bytes;
    for (size_t k = 0; k < lists.size(); ++k) {
        loff[k] = off;
        off += round16(lists[k].size() * sizeof(BItem));
    }
    B->args_off = off;
    const size_t total = off + args.size();
    cudaError_t e = dev_malloc(&B->dev, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        B->dev = nullptr;
        return bfail(B, FEWHA_ERR_OOM, "batch allocation failed");
    }
    unsigned char* base = static_cast<unsigned char*>(B->dev);
    BCK(cudaMemcpy(base, inst.data(), sizeof(BInst<T>) * n, cudaMemcpyHostToDevice), "batch upload");
    for (size_t k = 0; k < lists.size(); ++k)
        if (!lists[k].empty())
            BCK(cudaMemcpy(base + loff[k], lists[k].data(), lists[k].size() * sizeof(BItem), cudaMemcpyHostToDevice),
                "batch upload");
    BCK(cudaMemcpy(base + B->args_off, args.data(), args.size(), cudaMemcpyHostToDevice), "batch upload");
    B->args_host = args;
    // shared memory per (group, kind) and its limit
    const size_t S = recs[0].steps.size();
    std::vector<size_t> smem(G * BK_COUNT, 0);
    for (int i = 0; i < n; ++i)
        for (int kind = 0; kind < BK_COUNT; ++kind)
            smem[grp[i] * BK_COUNT + kind] = std::max(smem[grp[i] * BK_COUNT + kind], bsmem(B->h[i], kind));
    for (int kind = 0; kind < BK_COUNT; ++kind) {
        size_t lim = 0;
        BCK(batch_smem_limit<T>(kind, &lim), "batch smem attribute");
        for (int g = 0; g < G; ++g)
            if (bkind_list(kind) != BL_VEC && smem[g * BK_COUNT + kind] > lim)
                return bfail(B, FEWHA_ERR_LIMIT, "batched tile above the per-CTA shared-memory limit");
    }
    BCK(batch_set_taps(B->h[0]->setup.taps_h, B->h[0]->setup.taps_g), "batch taps");
    // launch shapes: projection CTA size, adjoint-projection taps, vector CTA size
    int kmax = 0;
    for (int i = 0; i < n; ++i) kmax = std::max(kmax, B->h[i]->kmax);
    const int pair_nt = cfg.pair_threads ? cfg.pair_threads : cblk<T>();
    const int taps = cfg.proj_taps ? cfg.proj_taps : (kmax <= 4 ? 4 : KMAX);
    const int vec_nt = cfg.vec_threads ? cfg.vec_threads : PBLK;
    if ((pair_nt != cblk<T>() && pair_nt != cblk<T>() / 2) || (taps != 4 && taps != KMAX) || taps < kmax ||
        (vec_nt != PBLK && vec_nt != 2 * PBLK))
        return bfail(B, FEWHA_ERR_INVALID_ARG, "launch shape not available for these instances");
    // capture
    BCK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal), "batch capture");
    cudaError_t le = cudaSuccess;
    if (G > 1) {
        le = cudaEventRecord(B->ev[0], B->cap);
        for (int g = 1; g < G && le == cudaSuccess; ++g) le = cudaStreamWaitEvent(B->branch[g], B->ev[0], 0);
    }
    for (int g = 0; g < G && le == cudaSuccess; ++g) {
        cudaStream_t st = g == 0 ? B->cap : B->branch[g];
        for (size_t j = 0; j < S && le == cudaSuccess; ++j) {
            const int kind = recs[0].steps[j].kind;
            const int li = g * BL_COUNT + bkind_list(kind);
            BLaunch L;
            L.kind = kind;
            L.inst = base;
            L.args = base + B->args_off + offs[j];
            L.items = reinterpret_cast<const BItem*>(base + loff[li]);
            L.n_items = static_cast<int>(lists[li].size());
            L.smem = smem[g * BK_COUNT + kind];
            L.pdl = (B->h[0]->params.flags & FEWHA_FLAG_PDL) != 0;
            L.pair_nt = pair_nt;
            L.taps = taps;
            L.vec_nt = vec_nt;
            le = batch_launch<T>(L, st);
        }
    }
    if (G > 1)
        for (int g = 1; g < G && le == cudaSuccess; ++g) {
            le = cudaEventRecord(B->ev[g], B->branch[g]);
            if (le == cudaSuccess) le = cudaStreamWaitEvent(B->cap, B->ev[g], 0);
        }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(B->cap, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bfail(B, FEWHA_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(le != cudaSuccess ? le : e));
    }
    e = cudaGraphInstantiate(&B->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        B->gexec = nullptr;
        return bfail(B, FEWHA_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    }
    B->have_plan = true;
    B->plan_warm = warm;
    B->plan_cfg = cfg;
    for (int i = 0; i < n; ++i) B->ver[i] = B->h[i]->version;
    return FEWHA_OK;
}

bool same_cfg(const fewha_batch_config& a, const fewha_batch_config& b) {
    return a.order == b.order && a.groups == b.groups && a.vec_passes == b.vec_passes &&
           a.pair_threads == b.pair_threads && a.proj_taps == b.proj_taps && a.vec_threads == b.vec_threads;
}

template <class T>
int batch_run(fewha_batch* B, const void* const* s_in, void* const* dm_in, void* stream) {
    if (!B) return FEWHA_ERR_INVALID_ARG;
    if (B->dead) return bfail(B, FEWHA_ERR_INVALID_ARG, "a member of the batch was destroyed");
    if (static_cast<int>(sizeof(T) * 8) != B->precision)
        return bfail(B, FEWHA_ERR_INVALID_ARG, "element type does not match the batch's precision");
    if (!s_in || !dm_in) return bfail(B, FEWHA_ERR_INVALID_ARG, "null pointer table");
    DeviceGuard g(B->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n = B->h.size();
    bool warm = false;
    for (size_t i = 0; i < n; ++i) {
        const fewha_handle* H = B->h[i];
        const bool w = (H->params.flags & FEWHA_FLAG_WARM_RESIDUAL) && H->have_prev;
        if (i == 0) warm = w;
        if (w != warm) return bfail(B, FEWHA_ERR_INVALID_ARG, "members differ in warm-residual state (reset them)");
    }
    const T* const* s = reinterpret_cast<const T* const*>(s_in);
    T* const* dm = reinterpret_cast<T* const*>(dm_in);
    std::vector<Recorder<T>> recs;
    int rc;
    if ((rc = batch_record<T>(B, s, dm, warm, recs))) return rc;
    std::vector<int> nparts(n);
    for (size_t i = 0; i < n; ++i) nparts[i] = bnparts(B->h[i], B->cfg.vec_passes, B->cfg.vec_threads);
    std::vector<unsigned char> args;
    std::vector<size_t> offs;
    batch_pack<T>(recs, nparts, args, offs);
    bool rebuild = !B->have_plan || B->plan_warm != warm || !same_cfg(B->plan_cfg, B->cfg) ||
                   args.size() != B->args_host.size();
    for (size_t i = 0; i < n && !rebuild; ++i) rebuild = B->ver[i] != B->h[i]->version;
    if (rebuild) {
        if ((rc = batch_build<T>(B, recs, nparts, args, offs, warm))) return rc;
    } else if (args != B->args_host) {
        B->args_host = args;
        BCK(cudaMemcpyAsync(static_cast<unsigned char*>(B->dev) + B->args_off, B->args_host.data(), args.size(),
                            cudaMemcpyHostToDevice, st),
            "batch arguments");
    }
    BCK(cudaGraphLaunch(B->gexec, st), "batch graph launch");
    for (size_t i = 0; i < n; ++i) B->h[i]->have_prev = true;
    return FEWHA_OK;
}

std::mutex g_tune_mutex;
std::vector<std::pair<std::string, fewha_batch_config>> g_tuned;   // shape signature -> config

std::string batch_signature(const fewha_batch* B) {
    std::string k = std::to_string(B->precision);
    for (const fewha_handle* H : B->h) {
        k += "|" + std::to_string(H->params.iters) + ":" + std::to_string(H->setup.n_act);
        for (const auto& L : H->setup.L) k += "," + std::to_string(L.n);
        k += ";";
        for (const auto& W : H->setup.G) k += "," + std::to_string(W.N);
    }
    return k;
}

template <class T>
int batch_autotune(fewha_batch* B, const void* const* s, void* const* dm, int reps, float* best_us, void* stream) {
    if (!B) return FEWHA_ERR_INVALID_ARG;
    if (B->dead) return bfail(B, FEWHA_ERR_INVALID_ARG, "a member of the batch was destroyed");
    if (reps < 1 || reps > 10000) return bfail(B, FEWHA_ERR_INVALID_ARG, "reps out of range");
    DeviceGuard g(B->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n = B->h.size();
    // snapshot of the warm state
    size_t per = 0;
    for (const fewha_handle* H : B->h) per += (3 * static_cast<size_t>(H->setup.n_c) + H->setup.n_act) * sizeof(T);
    void* snap = nullptr;
    if (dev_malloc(&snap, per) != cudaSuccess) {
        cudaGetLastError();
        return bfail(B, FEWHA_ERR_OOM, "autotune snapshot allocation failed");
    }
    std::vector<bool> had(n);
    auto copy_state = [&](bool save) {
        unsigned char* p = static_cast<unsigned char*>(snap);
        for (size_t i = 0; i < n; ++i) {
            fewha_handle* H = B->h[i];
            void* v[4] = {H->c, H->r, H->b_prev, H->a_prev};
            const size_t sz[4] = {H->setup.n_c * sizeof(T), H->setup.n_c * sizeof(T), H->setup.n_c * sizeof(T),
                                  H->setup.n_act * sizeof(T)};
            for (int k = 0; k < 4; ++k) {
                cudaMemcpyAsync(save ? p : v[k], save ? v[k] : p, sz[k], cudaMemcpyDeviceToDevice, st);
                p += sz[k];
            }
            if (save) had[i] = H->have_prev;
            else H->have_prev = had[i];
        }
    };
    copy_state(true);
    const fewha_batch_config start = B->cfg;
    fewha_batch_config best = start;
    float best_t = -1.f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = FEWHA_OK;
    // time one candidate (two untimed frames first: the plan is rebuilt for a new shape)
    auto trial = [&](const fewha_batch_config& c) {
        B->cfg = c;
        for (int w = 0; w < 2 && rc == FEWHA_OK; ++w) rc = batch_run<T>(B, s, dm, stream);
        if (rc) return;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && rc == FEWHA_OK; ++r) rc = batch_run<T>(B, s, dm, stream);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = bfail(B, FEWHA_ERR_CUDA, "autotune timing");
        if (rc) return;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const float us = 1e3f * ms / reps;
        if (best_t < 0.f || us < best_t) {
            best_t = us;
            best = c;
        }
    };
    // stage 1: work order, launch chains and vector passes with the default kernel shapes
    const int groups[] = {1, 2, 4, 8};
    const int vps[] = {1, 4};
    for (int order = 0; order < 2 && rc == FEWHA_OK; ++order)
        for (int gi = 0; gi < 4 && rc == FEWHA_OK; ++gi) {
            if (groups[gi] > static_cast<int>(n)) continue;
            for (int vi = 0; vi < 2 && rc == FEWHA_OK; ++vi) trial(fewha_batch_config{order, groups[gi], vps[vi], 0, 0, 0});
        }
    // stage 2: from the best of stage 1, the kernels' launch shapes
    int kmax = 0;
    for (const fewha_handle* H : B->h) kmax = std::max(kmax, H->kmax);
    const int nt = cblk<T>();
    const fewha_batch_config base = best;
    for (int pt : {nt, nt / 2})
        for (int tp : {4, KMAX})
            for (int vt : {PBLK, 2 * PBLK}) {
                if (rc != FEWHA_OK || tp < kmax) continue;
                fewha_batch_config c = base;
                c.pair_threads = pt;
                c.proj_taps = tp;
                c.vec_threads = vt;
                trial(c);
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    copy_state(false);
    const cudaError_t se = cudaStreamSynchronize(st);
    cudaFree(snap);
    if (rc) {
        B->cfg = start;
        return rc;
    }
    if (se != cudaSuccess) return bfail(B, FEWHA_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(se));
    B->cfg = best;
    if (best_us) *best_us = best_t;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    const std::string key = batch_signature(B);
    bool found = false;
    for (auto& kv : g_tuned)
        if (kv.first == key) {
            kv.second = best;
            found = true;
        }
    if (!found) g_tuned.emplace_back(key, best);
    return FEWHA_OK;
}

void batch_free(fewha_batch* B) {
    if (!B) return;
    DeviceGuard g(B->device);
    cudaDeviceSynchronize();
    batch_drop_plan(B);
    for (fewha_handle* H : B->h)
        if (H) H->batches.erase(std::remove(H->batches.begin(), H->batches.end(), B), H->batches.end());
    if (B->cap) cudaStreamDestroy(B->cap);
    for (int g2 = 0; g2 < FEWHA_BATCH_MAX_GROUPS; ++g2) {
        if (B->branch[g2]) cudaStreamDestroy(B->branch[g2]);
        if (B->ev[g2]) cudaEventDestroy(B->ev[g2]);
    }
    delete B;
}

int batch_create(fewha_handle* const* hs, int count, fewha_batch** out) {
    if (!out) return FEWHA_ERR_INVALID_ARG;
    *out = nullptr;
    if (!hs || count < 1 || count > FEWHA_BATCH_MAX_COUNT) return FEWHA_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        if (!hs[i]) return FEWHA_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(hs[i], FEWHA_ERR_INVALID_ARG, "a handle appears twice in a batch");
        if (hs[i]->device != hs[0]->device || hs[i]->precision != hs[0]->precision)
            return fail(hs[i], FEWHA_ERR_INVALID_ARG, "batch members differ in device or precision");
    }
    fewha_batch* B = new fewha_batch();
    B->h.assign(hs, hs + count);
    B->ver.assign(count, 0);
    B->precision = hs[0]->precision;
    B->device = hs[0]->device;
    DeviceGuard g(B->device);
    bool ok = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) == cudaSuccess;
    for (int g2 = 0; g2 < FEWHA_BATCH_MAX_GROUPS && ok; ++g2) {
        ok = cudaStreamCreateWithFlags(&B->branch[g2], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&B->ev[g2], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        B->h.clear();
        batch_free(B);
        return FEWHA_ERR_CUDA;
    }
    for (fewha_handle* H : B->h) H->batches.push_back(B);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        const std::string key = batch_signature(B);
        for (const auto& kv : g_tuned)
            if (kv.first == key) B->cfg = kv.second;
    }
    *out = B;
    return FEWHA_OK;
}

std::mutex g_registry_mutex;
std::vector<fewha_batch*> g_registry;   // batches of fewha_reconstruct_batched

template <class T>
int reconstruct_batched(fewha_handle* const* hs, int count, const T* const* s, T* const* dm, void* stream) {
    if (!hs || count < 1 || count > FEWHA_BATCH_MAX_COUNT) return FEWHA_ERR_INVALID_ARG;
    fewha_batch* B = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_registry_mutex);
        for (fewha_batch* b : g_registry)
            if (!b->dead && static_cast<int>(b->h.size()) == count && std::equal(b->h.begin(), b->h.end(), hs)) B = b;
    }
    if (!B) {
        const int rc = batch_create(hs, count, &B);
        if (rc) return rc;
        B->registry = true;
        std::lock_guard<std::mutex> lk(g_registry_mutex);
        g_registry.push_back(B);
    }
    const int rc = batch_run<T>(B, reinterpret_cast<const void* const*>(s), reinterpret_cast<void* const*>(dm), stream);
    if (rc) fail(hs[0], rc, B->err);
    return rc;
}

// A member handle is being destroyed: cached batches go, user batches are disabled.
void batches_forget(fewha_handle* H) {
    std::vector<fewha_batch*> bs = H->batches;
    for (fewha_batch* B : bs) {
        B->dead = true;
        for (auto& m : B->h)
            if (m == H) m = nullptr;
        if (B->registry) {
            {
                std::lock_guard<std::mutex> lk(g_registry_mutex);
                g_registry.erase(std::remove(g_registry.begin(), g_registry.end(), B), g_registry.end());
            }
            batch_free(B);
        }
    }
    H->batches.clear();
}

// ---------------------------------------------------------------- operators
template <class T>
int op_dispatch(fewha_handle* H, int op, const void* in, void* out, int iters, cudaStream_t st) {
    const Desc<T> d = make_desc<T>(H);
    const T* x = static_cast<const T*>(in);
    T* y = static_cast<T*>(out);
    T* u = static_cast<T*>(H->u);
    T* phi = static_cast<T*>(H->phi);
    int rc = 0;
    switch (op) {
        case 0:  // M
            return enqueue_apply<T>(H, d, x, y, PQ_SCRATCH_SLOT, false, st);
        case 1:  // rhs
            return enqueue_rhs<T>(H, d, x, y, st);
        case 2:  // dwt
            return launch_layer<T, LSRC_PHI, LDST_COEF, false>(H, d, layer_args<T>(H, x, y), st);
        case 3:  // idwt
            return launch_layer<T, LSRC_COEF, LDST_PHI, false>(H, d, layer_args<T>(H, x, y), st);
        case 4:  // project
            return launch_sensor<T, SSRC_PHI, false, SDST_NODES>(H, d, x, y, st);
        case 5:  // project adjoint
            return launch_layer<T, LSRC_NODES, LDST_PHI, false>(H, d, layer_args<T>(H, x, y), st);
        case 6:  // slopes
            return launch_sensor<T, SSRC_NODES, false, SDST_SLOPES>(H, d, x, y, st);
        case 7:  // slopes adjoint
            return launch_sensor<T, SSRC_SLOPES, false, SDST_ADJ>(H, d, x, y, st);
        case 8:  // noise weight
            return launch_sensor<T, SSRC_SLOPES, true, SDST_SLOPES>(H, d, x, y, st);
        case 9:  // forward model
            return launch_sensor<T, SSRC_PHI, false, SDST_SLOPES>(H, d, x, y, st);
        case 10:  // forward adjoint
            if ((rc = launch_sensor<T, SSRC_SLOPES, false, SDST_ADJ>(H, d, x, u, st))) return rc;
            return launch_layer<T, LSRC_NODES, LDST_PHI, false>(H, d, layer_args<T>(H, u, y), st);
        case 11:  // fit
            return enqueue_fit<T>(H, d, x, y, false, st);
        case 12:  // fit adjoint
            return launch_layer<T, LSRC_DM, LDST_COEF, false>(H, d, layer_args<T>(H, x, y), st);
        case 13: {  // pcg on b = in, c = out (in/out)
            CK(cudaMemcpyAsync(H->b, x, d.n_c * sizeof(T), cudaMemcpyDeviceToDevice, st), "b copy");
            return enqueue_pcg<T>(H, d, y, iters, false, st);
        }
        default:
            (void)phi;
            return fail(H, FEWHA_ERR_INVALID_ARG, "unknown operator");
    }
}

// Back-to-back launches of one hot-path kernel on the internal buffers (timing only).
template <class T>
int bench_stage(fewha_handle* H, int stage, int reps, cudaStream_t st) {
    const Desc<T> d = make_desc<T>(H);
    T* p = static_cast<T*>(H->p);
    T* phi = static_cast<T*>(H->phi);
    T* u = static_cast<T*>(H->u);
    T* q = static_cast<T*>(H->q);
    int rc = 0;
    for (int i = 0; i < reps && rc == 0; ++i) {
        switch (stage) {
            case FEWHA_STAGE_IDWT: {
                ClArgs<T> a = cl_args<T>(H, p, phi);
                a.pupd = p;
                a.zupd = static_cast<const T*>(H->z);
                a.iter = 1;
                a.zero_piston = 1;
                rc = launch_inv<T, 1>(H, d, a, st);
                break;
            }
            case FEWHA_STAGE_SENSOR:
                rc = launch_csensor<T, SSRC_PHI>(H, d, phi, u, st);
                break;
            case FEWHA_STAGE_LAYER: {
                ClArgs<T> a = cl_args<T>(H, u, q);
                a.pin = p;
                a.iter = PQ_SCRATCH_SLOT;
                a.zero_piston = 1;
                rc = launch_fwd<T, LSRC_NODES, LDST_APPLY>(H, d, a, st);
                break;
            }
            case FEWHA_STAGE_VECTOR:
                rc = launch_vec<T, V_UPDATE>(H, d.n_c, vec_args<T>(H, static_cast<T*>(H->c), 0), st);
                break;
            case FEWHA_STAGE_RHS:
                rc = launch_csensor<T, SSRC_SLOPES>(H, d, static_cast<const T*>(H->s_tmp), u, st);
                break;
            case FEWHA_STAGE_FIT:
                rc = launch_fit<T>(H, d, phi, static_cast<T*>(H->a_prev), static_cast<T*>(H->dm_tmp), 1, st);
                break;
            case FEWHA_STAGE_PROJ:
                rc = launch_proj<T>(H, d, phi, st);
                break;
            case FEWHA_STAGE_PROJT:
                rc = launch_projT<T>(H, d, u, st);
                break;
        }
    }
    return rc;
}

int op_entry(fewha_handle* H, int op, const void* in, void* out, int iters, void* stream) {
    if (!H) return FEWHA_ERR_INVALID_ARG;
    if (!in || !out) return fail(H, FEWHA_ERR_INVALID_ARG, "null pointer");
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return H->precision == 32 ? op_dispatch<float>(H, op, in, out, iters, st)
                              : op_dispatch<double>(H, op, in, out, iters, st);
}

// ---------------------------------------------------------------- no-allocation M-apply
// Scratch of fewha_apply_M_noalloc: a fixed 2 MiB block in this library's device image.
// Every GPU that loads the library holds it until the process exits.  In host code the
// name below is only a host-side stand-in: its device address comes from
// cudaGetSymbolAddress, taken once per device by noalloc_scratch().
static __device__ __align__(256) unsigned char fewha_noalloc_scratch[FEWHA_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[FEWHA_NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch block on the current device (set up on first use).
int noalloc_scratch(fewha_handle* H, unsigned char** out) {
    if (H->device < 0 || H->device >= FEWHA_NOALLOC_MAX_DEVICES)
        return fail(H, FEWHA_ERR_LIMIT, "fewha_apply_M_noalloc: device ordinal above the scratch table");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[H->device]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, fewha_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(H, e, "fewha_apply_M_noalloc: cudaGetSymbolAddress");
        g_noalloc_addr[H->device] = ptr;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[H->device]);
    return FEWHA_OK;
}

size_t round256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

template <class T>
int apply_M_noalloc(fewha_handle* H, const T* x, T* qout, cudaStream_t st) {
    const size_t b_phi = round256(static_cast<size_t>(H->setup.n_c) * sizeof(T));
    const size_t b_u = round256(static_cast<size_t>(H->setup.n_nodes) * sizeof(T));
    const size_t b_pq = round256(static_cast<size_t>(MAXL) * sizeof(double));
    const size_t need = b_phi + b_u + b_pq;
    if (need > FEWHA_NOALLOC_SCRATCH_BYTES)
        return fail(H, FEWHA_ERR_LIMIT,
                    "fewha_apply_M_noalloc: this instance needs " + std::to_string(need) +
                        " bytes of scratch, more than the " +
                        std::to_string(static_cast<size_t>(FEWHA_NOALLOC_SCRATCH_BYTES)) +
                        "-byte static block; use fewha_apply_M");
    unsigned char* base = nullptr;
    int rc = noalloc_scratch(H, &base);
    if (rc) return rc;
    T* phi = reinterpret_cast<T*>(base);
    T* u = reinterpret_cast<T*>(base + b_phi);
    // the layer kernel also writes each layer's p.q partial; nothing reads them in this
    // entry point, so these slots are write-only and need no clearing
    double* pq = reinterpret_cast<double*>(base + b_phi + b_u);
    const Desc<T> d = make_desc<T>(H);
    if ((rc = launch_layer<T, LSRC_COEF, LDST_PHI, false>(H, d, layer_args<T>(H, x, phi), st))) return rc;
    if ((rc = launch_sensor<T, SSRC_PHI, true, SDST_ADJ>(H, d, phi, u, st))) return rc;
    LayerArgs<T> a = layer_args<T>(H, u, qout);
    a.pin = x;
    a.iter = 0;
    a.zero_piston = 1;
    a.pcg.pqpart = pq;
    return launch_layer<T, LSRC_NODES, LDST_APPLY, false>(H, d, a, st);
}

}  // namespace

// =====================================================================================
extern "C" {

const char* fewha_create_error(void) { return g_create_error.c_str(); }

const char* fewha_last_error(const fewha_handle* h) { return h ? h->err.c_str() : "null handle"; }

int fewha_create(const fewha_telescope* tel, const fewha_wfs* wfs, int n_wfs, const fewha_layer* layers,
                 int n_layers, const fewha_dm* dms, int n_dms, const fewha_params* params,
                 fewha_handle** out) {
    FEWHA_RANGE("fewha_create");
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return FEWHA_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!tel) {
        g_create_error = "telescope is NULL";
        return FEWHA_ERR_INVALID_ARG;
    }
    int rc = check_params(params, g_create_error);
    if (rc) return rc;
    fewha_handle* H = new fewha_handle();
    H->params = *params;
    H->precision = params->precision;
    H->esz = params->precision == 32 ? sizeof(float) : sizeof(double);
    rc = build_setup(*tel, wfs, n_wfs, layers, n_layers, dms, n_dms, H->setup, g_create_error);
    if (!rc) set_elongation(H->setup, params->alpha_eta);
    if (!rc && (params->flags & FEWHA_FLAG_CLOSED_LOOP) && !H->setup.dm_proj_ok) {
        g_create_error = "closed loop needs every DM below every LGS";
        rc = FEWHA_ERR_GEOMETRY;
    }
    if (rc) {
        delete H;
        return rc;
    }
    for (int l = 0; l < n_layers; ++l) H->weights.push_back(layers[l].cn2_weight);
    H->tel_in = *tel;
    H->wfs_in.assign(wfs, wfs + n_wfs);
    H->layers_in.assign(layers, layers + n_layers);
    if (n_dms > 0) H->dms_in.assign(dms, dms + n_dms);
    H->npart = (H->setup.n_c + PBLK * 4 - 1) / (PBLK * 4);
    if (H->npart > NPART_MAX) H->npart = NPART_MAX;
    if (H->npart < 1) H->npart = 1;
    if (cudaGetDevice(&H->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "no usable CUDA device";
        free_handle(H);
        return FEWHA_ERR_CUDA;
    }
    rc = H->precision == 32 ? typed_create<float>(H) : typed_create<double>(H);
    if (rc) {
        g_create_error = H->err;
        free_handle(H);
        return rc;
    }
    *out = H;
    return FEWHA_OK;
}

void fewha_destroy(fewha_handle* h) {
    if (!h) return;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    batches_forget(h);
    free_handle(h);
}

int fewha_sizes(const fewha_handle* h, int64_t* n_slopes, int64_t* n_coeffs, int64_t* n_act,
                int64_t* n_nodes) {
    if (!h) return FEWHA_ERR_INVALID_ARG;
    if (n_slopes) *n_slopes = h->setup.n_s;
    if (n_coeffs) *n_coeffs = h->setup.n_c;
    if (n_act) *n_act = h->setup.n_act;
    if (n_nodes) *n_nodes = h->setup.n_nodes;
    return FEWHA_OK;
}

int fewha_update_params(fewha_handle* H, const fewha_params* params, const double* cn2_weights,
                        const double* sigmas) {
    FEWHA_RANGE("fewha_update_params");
    if (!H) return FEWHA_ERR_INVALID_ARG;
    std::string e;
    int rc = check_params(params, e);
    if (rc) return fail(H, rc, e);
    if (params->precision != H->precision) return fail(H, FEWHA_ERR_INVALID_ARG, "precision cannot change");
    if ((params->flags & FEWHA_FLAG_CLOSED_LOOP) && !H->setup.dm_proj_ok)
        return fail(H, FEWHA_ERR_GEOMETRY, "closed loop needs every DM below every LGS");
    DeviceGuard g(H->device);
    CK(cudaDeviceSynchronize(), "update sync");
    if (cn2_weights) {
        for (size_t l = 0; l < H->weights.size(); ++l) {
            if (!(cn2_weights[l] > 0)) return fail(H, FEWHA_ERR_INVALID_ARG, "Cn2 weights must be > 0");
            H->weights[l] = cn2_weights[l];
        }
    }
    if (sigmas) {
        for (size_t g2 = 0; g2 < H->setup.G.size(); ++g2) {
            if (!(sigmas[g2] > 0)) return fail(H, FEWHA_ERR_INVALID_ARG, "sigmas must be > 0");
            H->setup.G[g2].sig2inv = 1.0 / (sigmas[g2] * sigmas[g2]);
            H->setup.wfs_sigma[g2] = sigmas[g2];
        }
    }
    H->params = *params;
    set_elongation(H->setup, params->alpha_eta);
    drop_graph(H);
    H->have_prev = false;
    H->aug_m = 0;                     // M changed: the stored directions no longer apply
    ++H->version;
    H->grad_ready = false;
    rc = H->precision == 32 ? compute_diagonals<float>(H) : compute_diagonals<double>(H);
    if (rc || !H->twin) return rc;
    return twin_params(H);
}

int fewha_reset(fewha_handle* H, void* stream) {
    if (!H) return FEWHA_ERR_INVALID_ARG;
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaMemsetAsync(H->c, 0, H->setup.n_c * H->esz, st), "reset");
    CK(cudaMemsetAsync(H->a_prev, 0, H->setup.n_act * H->esz, st), "reset");
    CK(cudaMemsetAsync(H->r, 0, H->setup.n_c * H->esz, st), "reset");
    CK(cudaMemsetAsync(H->b_prev, 0, H->setup.n_c * H->esz, st), "reset");
    CK(cudaMemsetAsync(H->a_old, 0, H->setup.n_act * H->esz, st), "reset");
    H->have_prev = false;
    H->aug_m = 0;
    return FEWHA_OK;
}

int fewha_reconstruct(fewha_handle* h, const float* s, float* x, float* dm, void* stream) {
    FEWHA_RANGE("fewha_reconstruct");
    return reconstruct_dev<float>(h, s, x, dm, stream);
}
int fewha_reconstruct_f64(fewha_handle* h, const double* s, double* x, double* dm, void* stream) {
    FEWHA_RANGE("fewha_reconstruct_f64");
    return reconstruct_dev<double>(h, s, x, dm, stream);
}
int fewha_reconstruct_host(fewha_handle* h, const float* s, float* dm, void* stream) {
    FEWHA_RANGE("fewha_reconstruct_host");
    return reconstruct_host<float>(h, s, dm, stream);
}
int fewha_reconstruct_host_f64(fewha_handle* h, const double* s, double* dm, void* stream) {
    FEWHA_RANGE("fewha_reconstruct_host_f64");
    return reconstruct_host<double>(h, s, dm, stream);
}

int fewha_run_loop(fewha_handle* h, const float* s, int n_frames, float* dm, double period_us,
                   float* wall_us, float* device_us, int* n_late, void* stream) {
    FEWHA_RANGE("fewha_run_loop");
    return run_loop<float>(h, s, n_frames, dm, period_us, wall_us, device_us, n_late, stream);
}
int fewha_run_loop_f64(fewha_handle* h, const double* s, int n_frames, double* dm, double period_us,
                       float* wall_us, float* device_us, int* n_late, void* stream) {
    FEWHA_RANGE("fewha_run_loop_f64");
    return run_loop<double>(h, s, n_frames, dm, period_us, wall_us, device_us, n_late, stream);
}

int fewha_batch_create(fewha_handle* const* handles, int count, fewha_batch** out) {
    return batch_create(handles, count, out);
}
void fewha_batch_destroy(fewha_batch* b) {
    if (!b) return;
    if (b->registry) return;   // owned by the fewha_reconstruct_batched cache
    batch_free(b);
}
const char* fewha_batch_last_error(const fewha_batch* b) { return b ? b->err.c_str() : "null batch"; }
int fewha_batch_set_config(fewha_batch* b, const fewha_batch_config* cfg) {
    if (!b || !cfg) return FEWHA_ERR_INVALID_ARG;
    const int nt = b->precision == 32 ? cblk<float>() : cblk<double>();
    if (cfg->order < 0 || cfg->order > 1 || cfg->groups < 1 || cfg->groups > FEWHA_BATCH_MAX_GROUPS ||
        cfg->vec_passes < 1 || cfg->vec_passes > 8 ||
        (cfg->pair_threads != 0 && cfg->pair_threads != nt && cfg->pair_threads != nt / 2) ||
        (cfg->proj_taps != 0 && cfg->proj_taps != 4 && cfg->proj_taps != KMAX) ||
        (cfg->vec_threads != 0 && cfg->vec_threads != PBLK && cfg->vec_threads != 2 * PBLK))
        return bfail(b, FEWHA_ERR_INVALID_ARG, "configuration out of range");
    int kmax = 0;
    for (const fewha_handle* H : b->h)
        if (H) kmax = std::max(kmax, H->kmax);
    if (cfg->proj_taps != 0 && cfg->proj_taps < kmax)
        return bfail(b, FEWHA_ERR_INVALID_ARG, "proj_taps below the members' tap count");
    b->cfg = *cfg;
    return FEWHA_OK;
}
int fewha_batch_get_config(const fewha_batch* b, fewha_batch_config* cfg) {
    if (!b || !cfg) return FEWHA_ERR_INVALID_ARG;
    *cfg = b->cfg;
    return FEWHA_OK;
}
int fewha_batch_reconstruct(fewha_batch* b, const void* const* s, void* const* dm, void* stream) {
    FEWHA_RANGE("fewha_batch_reconstruct");
    if (!b) return FEWHA_ERR_INVALID_ARG;
    return b->precision == 32 ? batch_run<float>(b, s, dm, stream) : batch_run<double>(b, s, dm, stream);
}
int fewha_batch_autotune(fewha_batch* b, const void* const* s, void* const* dm, int reps, float* best_us,
                         void* stream) {
    if (!b) return FEWHA_ERR_INVALID_ARG;
    return b->precision == 32 ? batch_autotune<float>(b, s, dm, reps, best_us, stream)
                              : batch_autotune<double>(b, s, dm, reps, best_us, stream);
}
int fewha_reconstruct_batched(fewha_handle* const* hs, int count, const float* const* s, float* const* dm,
                              void* stream) {
    FEWHA_RANGE("fewha_reconstruct_batched");
    if (hs && count > 0 && hs[0] && hs[0]->precision != 32) return fail(hs[0], FEWHA_ERR_INVALID_ARG, "precision mismatch");
    return reconstruct_batched<float>(hs, count, s, dm, stream);
}
int fewha_reconstruct_batched_f64(fewha_handle* const* hs, int count, const double* const* s, double* const* dm,
                                  void* stream) {
    FEWHA_RANGE("fewha_reconstruct_batched_f64");
    if (hs && count > 0 && hs[0] && hs[0]->precision != 64) return fail(hs[0], FEWHA_ERR_INVALID_ARG, "precision mismatch");
    return reconstruct_batched<double>(hs, count, s, dm, stream);
}

int fewha_get_state(fewha_handle* H, void* c, void* a_prev, void* stream) {
    if (!H) return FEWHA_ERR_INVALID_ARG;
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (c) CK(cudaMemcpyAsync(c, H->c, H->setup.n_c * H->esz, cudaMemcpyDeviceToDevice, st), "get state");
    if (a_prev)
        CK(cudaMemcpyAsync(a_prev, H->a_prev, H->setup.n_act * H->esz, cudaMemcpyDeviceToDevice, st), "get state");
    return FEWHA_OK;
}

int fewha_set_state(fewha_handle* H, const void* c, const void* a_prev, void* stream) {
    if (!H) return FEWHA_ERR_INVALID_ARG;
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (c) CK(cudaMemcpyAsync(H->c, c, H->setup.n_c * H->esz, cudaMemcpyDeviceToDevice, st), "set state");
    if (a_prev)
        CK(cudaMemcpyAsync(H->a_prev, a_prev, H->setup.n_act * H->esz, cudaMemcpyDeviceToDevice, st), "set state");
    H->have_prev = false;
    H->aug_m = 0;
    return FEWHA_OK;
}

int fewha_get_residual(fewha_handle* H, void* r, void* b, void* stream) {
    if (!H) return FEWHA_ERR_INVALID_ARG;
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (r) CK(cudaMemcpyAsync(r, H->r, H->setup.n_c * H->esz, cudaMemcpyDeviceToDevice, st), "get residual");
    if (b) {
        // the plain explicit frame forms r0 from the slopes' residual and never forms b
        if (!(H->params.flags & (FEWHA_FLAG_WARM_RESIDUAL | FEWHA_FLAG_PERSISTENT)))
            return fail(H, FEWHA_ERR_INVALID_ARG, "this frame form does not form b (use fewha_rhs)");
        CK(cudaMemcpyAsync(b, H->b, H->setup.n_c * H->esz, cudaMemcpyDeviceToDevice, st), "get residual");
    }
    return FEWHA_OK;
}

int fewha_solve(fewha_handle* H, const void* b, void* x, double tol, int max_iters, int* iters,
                double* rel, void* stream) {
    FEWHA_RANGE("fewha_solve");
    if (!H) return FEWHA_ERR_INVALID_ARG;
    if (!b || !x || !(tol >= 0.0) || max_iters < 0) return fail(H, FEWHA_ERR_INVALID_ARG, "bad solve arguments");
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return H->precision == 32
               ? solve_entry<float>(H, static_cast<const float*>(b), static_cast<float*>(x), tol, max_iters, st,
                                    iters, rel)
               : solve_entry<double>(H, static_cast<const double*>(b), static_cast<double*>(x), tol, max_iters, st,
                                     iters, rel);
}

int fewha_reconstruct_converged(fewha_handle* H, const void* s, void* dm, double tol, int max_iters,
                                int* iters, double* rel, void* stream) {
    FEWHA_RANGE("fewha_reconstruct_converged");
    if (!H) return FEWHA_ERR_INVALID_ARG;
    if (!s || !dm || !(tol >= 0.0) || max_iters < 0) return fail(H, FEWHA_ERR_INVALID_ARG, "bad arguments");
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return H->precision == 32
               ? reconstruct_converged<float>(H, static_cast<const float*>(s), static_cast<float*>(dm), tol,
                                              max_iters, iters, rel, st)
               : reconstruct_converged<double>(H, static_cast<const double*>(s), static_cast<double*>(dm), tol,
                                               max_iters, iters, rel, st);
}

int fewha_backward(fewha_handle* H, const void* g_dm, void* g_s, double* g_alpha, double* g_cn2, void* stream) {
    FEWHA_RANGE("fewha_backward");
    if (!H) return FEWHA_ERR_INVALID_ARG;
    if (!g_dm) return fail(H, FEWHA_ERR_INVALID_ARG, "null gradient of the commands");
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return H->precision == 32
               ? backward<float>(H, static_cast<const float*>(g_dm), static_cast<float*>(g_s), g_alpha, g_cn2, st)
               : backward<double>(H, static_cast<const double*>(g_dm), static_cast<double*>(g_s), g_alpha, g_cn2,
                                  st);
}

int fewha_frame_vjp(fewha_handle* H, const void* s, const void* c0, const void* g_dm, void* dm, void* g_s,
                    void* stream) {
    FEWHA_RANGE("fewha_frame_vjp");
    if (!H) return FEWHA_ERR_INVALID_ARG;
    if (!s || !c0 || (g_dm && !g_s)) return fail(H, FEWHA_ERR_INVALID_ARG, "null slopes, warm start or gradient output");
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return H->precision == 32
               ? frame_vjp<float>(H, static_cast<const float*>(s), static_cast<const float*>(c0),
                                  static_cast<const float*>(g_dm), static_cast<float*>(dm), static_cast<float*>(g_s), st)
               : frame_vjp<double>(H, static_cast<const double*>(s), static_cast<const double*>(c0),
                                   static_cast<const double*>(g_dm), static_cast<double*>(dm),
                                   static_cast<double*>(g_s), st);
}

int fewha_check_input(fewha_handle* H, int* nonfinite, void* stream) {
    if (!H || !nonfinite) return FEWHA_ERR_INVALID_ARG;
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned flag = 0;
    CK(cudaMemcpyAsync(&flag, H->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "status");
    CK(cudaMemsetAsync(H->status, 0, sizeof(unsigned), st), "status");
    CK(cudaStreamSynchronize(st), "status");
    *nonfinite = (flag & 1u) ? 1 : 0;
    if (flag & 2u) return fail(H, FEWHA_ERR_TIMEOUT, "a grid-wide wait of the persistent frame ran out");
    return FEWHA_OK;
}

int fewha_apply_M(fewha_handle* h, const void* c, void* q, void* st) { return op_entry(h, 0, c, q, 0, st); }
int fewha_rhs(fewha_handle* h, const void* s, void* b, void* st) { return op_entry(h, 1, s, b, 0, st); }
int fewha_dwt(fewha_handle* h, const void* phi, void* c, void* st) { return op_entry(h, 2, phi, c, 0, st); }
int fewha_idwt(fewha_handle* h, const void* c, void* phi, void* st) { return op_entry(h, 3, c, phi, 0, st); }
int fewha_project(fewha_handle* h, const void* phi, void* v, void* st) { return op_entry(h, 4, phi, v, 0, st); }
int fewha_project_adj(fewha_handle* h, const void* v, void* phi, void* st) { return op_entry(h, 5, v, phi, 0, st); }
int fewha_slopes(fewha_handle* h, const void* v, void* s, void* st) { return op_entry(h, 6, v, s, 0, st); }
int fewha_slopes_adj(fewha_handle* h, const void* s, void* v, void* st) { return op_entry(h, 7, s, v, 0, st); }
int fewha_noise_weight(fewha_handle* h, const void* s, void* o, void* st) { return op_entry(h, 8, s, o, 0, st); }
int fewha_forward(fewha_handle* h, const void* phi, void* s, void* st) { return op_entry(h, 9, phi, s, 0, st); }
int fewha_forward_adj(fewha_handle* h, const void* s, void* phi, void* st) { return op_entry(h, 10, s, phi, 0, st); }
int fewha_fit(fewha_handle* h, const void* c, void* dm, void* st) { return op_entry(h, 11, c, dm, 0, st); }
int fewha_fit_adj(fewha_handle* h, const void* dm, void* c, void* st) { return op_entry(h, 12, dm, c, 0, st); }
int fewha_pcg(fewha_handle* h, const void* b, void* c, int iters, void* st) {
    if (h && (iters < 0 || iters > FEWHA_MAX_ITERS)) return fail(h, FEWHA_ERR_LIMIT, "iters out of range");
    return op_entry(h, 13, b, c, iters, st);
}

int fewha_fit_ls(fewha_handle* H, const fewha_lsfit* cfg, const void* c, void* dm, double tol, int max_iters,
                 int* iters, double* rel, void* stream) {
    FEWHA_RANGE("fewha_fit_ls");
    if (!H) return FEWHA_ERR_INVALID_ARG;
    if (!c || !dm || !(tol >= 0.0) || max_iters < 0) return fail(H, FEWHA_ERR_INVALID_ARG, "bad fit_ls arguments");
    int rc = check_lsfit(H, cfg);
    if (rc) return rc;
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return H->precision == 32
               ? fit_ls<float>(H, *cfg, static_cast<const float*>(c), static_cast<float*>(dm), tol, max_iters,
                               iters, rel, st)
               : fit_ls<double>(H, *cfg, static_cast<const double*>(c), static_cast<double*>(dm), tol, max_iters,
                                iters, rel, st);
}

int fewha_bench_stage(fewha_handle* H, int stage, int reps, void* stream) {
    if (!H) return FEWHA_ERR_INVALID_ARG;
    if (stage < 0 || stage >= FEWHA_NUM_STAGES || reps < 1)
        return fail(H, FEWHA_ERR_INVALID_ARG, "bad stage or repetition count");
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return H->precision == 32 ? bench_stage<float>(H, stage, reps, st)
                              : bench_stage<double>(H, stage, reps, st);
}

int fewha_frame_launches(const fewha_handle* H, int* launches) {
    if (!H || !launches) return FEWHA_ERR_INVALID_ARG;
    const bool warm = (H->params.flags & FEWHA_FLAG_WARM_RESIDUAL) != 0;
    // the plain explicit frame: r0 from the slopes' residual, 5 (the right-hand side is not
    // formed); with the warm recurrence, RHS 3 and r0 1 (its explicit refresh frames: 3 + 5);
    // augmented: r0 5 and one more start kernel (its direction update is fused into the
    // inverse kernel of each apply); 6 per iteration
    const int aug = (H->params.flags & FEWHA_FLAG_AUGMENTED) ? 1 : 0;
    const int closed = (H->params.flags & FEWHA_FLAG_CLOSED_LOOP) ? 2 : 0;
    // fit: 2 (inverse transform, fit), or 1 where the plain explicit frame carries the
    // layers of c through its iterations
    const int per_iter = 6, start = warm ? 3 + 1 : (aug ? 5 + 1 : 5);
    const int fit = (warm || aug) ? 2 : 1;
    *launches = (H->params.flags & FEWHA_FLAG_PERSISTENT) ? 1 : closed + start + aug + per_iter * H->params.iters + fit;
    return FEWHA_OK;
}

int fewha_device_bytes(const fewha_handle* H, int64_t* bytes) {
    if (!H || !bytes) return FEWHA_ERR_INVALID_ARG;
    int64_t total = 0;
    for (const fewha_handle* X = H; X; X = X->twin)
        for (size_t b : X->alloc_sizes) total += static_cast<int64_t>(b);
    *bytes = total;
    return FEWHA_OK;
}

int fewha_test_fail_alloc(int after) {
    g_fail_countdown = after < 0 ? -1 : after;
    return FEWHA_OK;
}

int fewha_set_wait_limit(fewha_handle* H, unsigned polls, unsigned extra) {
    if (!H) return FEWHA_ERR_INVALID_ARG;
    H->wait_limit = polls;
    H->wait_extra = extra;
    drop_graph(H);                    // the limits are kernel arguments of a captured frame
    return FEWHA_OK;
}

int fewha_get_diagonals(fewha_handle* H, void* d_D, void* d_J, void* stream) {
    if (!H) return FEWHA_ERR_INVALID_ARG;
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = H->setup.n_c;
    if (d_D) CK(cudaMemcpyAsync(d_D, H->D, n * H->esz, cudaMemcpyDeviceToDevice, st), "D copy");
    if (d_J) {
        if (H->precision == 64) {
            CK(cudaMemcpyAsync(d_J, H->J64, n * sizeof(double), cudaMemcpyDeviceToDevice, st), "J copy");
        } else {
            k_convert<float, double><<<(n + 255) / 256, 256, 0, st>>>(n, H->J64, static_cast<float*>(d_J));
            CK(cudaGetLastError(), "J convert");
        }
    }
    return FEWHA_OK;
}

int fewha_apply_M_noalloc(fewha_handle* H, const void* d_c, void* d_q, void* stream) {
    if (!H) return FEWHA_ERR_INVALID_ARG;
    if (!d_c || !d_q) return fail(H, FEWHA_ERR_INVALID_ARG, "fewha_apply_M_noalloc: null pointer");
    DeviceGuard g(H->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return H->precision == 32
               ? apply_M_noalloc<float>(H, static_cast<const float*>(d_c), static_cast<float*>(d_q), st)
               : apply_M_noalloc<double>(H, static_cast<const double*>(d_c), static_cast<double*>(d_q), st);
}

}  // extern "C"
