// Batched kernels: thin wrappers that run the single-instance kernel bodies on work items
// of many instances in one launch.  A CTA first copies its instance's descriptor into
// shared memory (the bodies then read it from there, as the single-instance kernels read
// theirs from the constant bank), then runs the body on its unit.
#include <algorithm>
#include <utility>

#include "fewha_batch.h"

namespace fewha {

namespace {

// Copy the leading desc_bytes of the instance's descriptor into shared memory.
template <class T>
__device__ __forceinline__ void load_desc(Desc<T>& sd, const BInst<T>* __restrict__ I) {
    const int4* src = reinterpret_cast<const int4*>(&I->d);
    int4* dst = reinterpret_cast<int4*>(&sd);
    const int nb = (I->desc_bytes + 15) >> 4;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

template <class T, int PUPD>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(cblk<T>(), 1)
    kb_cl_inv(const BInst<T>* __restrict__ inst, const ClArgs<T>* __restrict__ args,
              const BItem* __restrict__ items) {
    __shared__ __align__(16) Desc<T> sd;
    pdl_enter();
    const BItem it = items[blockIdx.y];
    const BInst<T>* I = inst + it.inst;
    load_desc<T>(sd, I);
    const ClArgs<T> a = args[it.inst];
    const ClLayout lay = I->lay_inv;
    cl_inv_body<T, PUPD>(sd, a, lay, it.unit);
}

template <class T, int DST>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(cblk<T>(), 1)
    kb_cl_fwd(const BInst<T>* __restrict__ inst, const ClArgs<T>* __restrict__ args,
              const BItem* __restrict__ items) {
    __shared__ __align__(16) Desc<T> sd;
    pdl_enter();
    const BItem it = items[blockIdx.y];
    const BInst<T>* I = inst + it.inst;
    load_desc<T>(sd, I);
    const ClArgs<T> a = args[it.inst];
    const ClLayout lay = I->lay_fwd;
    const PairBufs<T> pb = I->pb;
    cl_fwd_body<T, LSRC_NODES, DST>(sd, a, lay, pb, it.unit, I->ctas_layer);
}

template <class T, int SRC>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(cblk<T>(), 1)
    kb_cl_sensor(const BInst<T>* __restrict__ inst, const SensorArgs<T>* __restrict__ args,
                 const BItem* __restrict__ items) {
    __shared__ __align__(16) Desc<T> sd;
    pdl_enter();
    const BItem it = items[blockIdx.y];
    const BInst<T>* I = inst + it.inst;
    load_desc<T>(sd, I);
    const SensorArgs<T> a = args[it.inst];
    const SensorLayout lay = I->lay_sen;
    const PairBufs<T> pb = I->pb;
    cl_sensor_body<T, SRC>(sd, a, lay, pb, it.unit);
}

template <class T, int NTP>
__global__ void __launch_bounds__(NTP, 1)
    kb_proj(const BInst<T>* __restrict__ inst, const T* const* __restrict__ args,
            const BItem* __restrict__ items) {
    __shared__ __align__(16) Desc<T> sd;
    pdl_enter();
    const BItem it = items[blockIdx.x];
    const BInst<T>* I = inst + it.inst;
    load_desc<T>(sd, I);
    const PairBufs<T> pb = I->pb;
    proj_body<T, NTP>(sd, args[it.inst], pb, it.unit / MAXL, it.unit % MAXL);
}

template <class T, int KM, int NTP>
__global__ void __launch_bounds__(NTP, 1)
    kb_projT(const BInst<T>* __restrict__ inst, const T* const* __restrict__ args,
             const BItem* __restrict__ items) {
    __shared__ __align__(16) Desc<T> sd;
    pdl_enter();
    const BItem it = items[blockIdx.x];
    const BInst<T>* I = inst + it.inst;
    load_desc<T>(sd, I);
    const PairBufs<T> pb = I->pb;
    projT_body<T, KM, NTP>(sd, args[it.inst], pb, it.unit / MAXL, it.unit % MAXL);
}

template <class T, int PHASE, int NTV>
__global__ void __launch_bounds__(NTV)
    kb_vec(const BInst<T>* __restrict__ inst, const VecArgs<T>* __restrict__ args,
           const BItem* __restrict__ items) {
    pdl_enter();
    const BItem it = items[blockIdx.x];
    const BInst<T>* I = inst + it.inst;
    const VecArgs<T> v = args[it.inst];
    vec_body<T, PHASE, NTV>(I->d.n_c, v, it.unit, I->nparts);
}

template <class T>
__global__ void __launch_bounds__(PBLK)
    kb_fit(const BInst<T>* __restrict__ inst, const FitArgs<T>* __restrict__ args,
           const BItem* __restrict__ items) {
    __shared__ __align__(16) Desc<T> sd;
    pdl_enter();
    const BItem it = items[blockIdx.x];
    const BInst<T>* I = inst + it.inst;
    load_desc<T>(sd, I);
    const FitArgs<T> f = args[it.inst];
    fit_body<T>(sd, f.phi, f.a_prev, f.out, f.apply_gain, it.unit, nullptr, f.cpist);
}

// The kernel of a step kind in one launch shape (variant v: bit 0 half-size projection
// CTAs, bit 1 the 4-tap adjoint projection; for the vector kernels, bit 0 512 threads).
template <class T>
const void* kernel_of(int kind, int v) {
    constexpr int NP = cblk<T>(), NH = cblk<T>() / 2;
    const bool half = (v & 1) != 0, t4 = (v & 2) != 0;
    switch (kind) {
        case BK_INV: return reinterpret_cast<const void*>(kb_cl_inv<T, 0>);
        case BK_INV_UPD: return reinterpret_cast<const void*>(kb_cl_inv<T, 1>);
        case BK_PROJ:
            return half ? reinterpret_cast<const void*>(kb_proj<T, NH>) : reinterpret_cast<const void*>(kb_proj<T, NP>);
        case BK_SEN_PHI: return reinterpret_cast<const void*>(kb_cl_sensor<T, SSRC_PHI>);
        case BK_SEN_SLOPES: return reinterpret_cast<const void*>(kb_cl_sensor<T, SSRC_SLOPES>);
        case BK_SEN_RESID: return reinterpret_cast<const void*>(kb_cl_sensor<T, SSRC_RESID>);
        case BK_PROJT:
            if (t4)
                return half ? reinterpret_cast<const void*>(kb_projT<T, 4, NH>)
                            : reinterpret_cast<const void*>(kb_projT<T, 4, NP>);
            return half ? reinterpret_cast<const void*>(kb_projT<T, KMAX, NH>)
                        : reinterpret_cast<const void*>(kb_projT<T, KMAX, NP>);
        case BK_FWD_APPLY: return reinterpret_cast<const void*>(kb_cl_fwd<T, LDST_APPLY>);
        case BK_FWD_COEF: return reinterpret_cast<const void*>(kb_cl_fwd<T, LDST_COEF>);
        case BK_FWD_RINIT: return reinterpret_cast<const void*>(kb_cl_fwd<T, LDST_RESID_INIT>);
        case BK_VEC_INIT:
            return half ? reinterpret_cast<const void*>(kb_vec<T, V_INIT, 2 * PBLK>)
                        : reinterpret_cast<const void*>(kb_vec<T, V_INIT, PBLK>);
        case BK_VEC_WARM:
            return half ? reinterpret_cast<const void*>(kb_vec<T, V_INIT_WARM, 2 * PBLK>)
                        : reinterpret_cast<const void*>(kb_vec<T, V_INIT_WARM, PBLK>);
        case BK_VEC_UPDATE:
            return half ? reinterpret_cast<const void*>(kb_vec<T, V_UPDATE, 2 * PBLK>)
                        : reinterpret_cast<const void*>(kb_vec<T, V_UPDATE, PBLK>);
        case BK_FIT: return reinterpret_cast<const void*>(kb_fit<T>);
        default: return nullptr;
    }
}

}  // namespace

cudaError_t batch_set_taps(const double* h, const double* g) {
    float h32[6], g32[6];
    for (int k = 0; k < 6; ++k) {
        h32[k] = static_cast<float>(h[k]);
        g32[k] = static_cast<float>(g[k]);
    }
    cudaError_t e = cudaMemcpyToSymbol(c_h32, h32, sizeof(h32));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_g32, g32, sizeof(g32));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_h64, h, 6 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_g64, g, 6 * sizeof(double));
    return e;
}

template <class T>
cudaError_t batch_smem_limit(int kind, size_t* bytes) {
    if (bkind_list(kind) == BL_VEC) {
        *bytes = 0;
        return cudaSuccess;
    }
    int lim = 227 * 1024;
    for (int v = 0; v < 4; ++v) {
        const void* k = kernel_of<T>(kind, v);
        if (!k) return cudaErrorInvalidValue;
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k);
        if (e != cudaSuccess) return e;
        const int avail = 227 * 1024 - static_cast<int>(fa.sharedSizeBytes);
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, avail)) != cudaSuccess) return e;
        lim = std::min(lim, avail);
    }
    *bytes = static_cast<size_t>(lim);
    return cudaSuccess;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_b(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <class T>
cudaError_t batch_launch(const BLaunch& L, cudaStream_t st) {
    if (L.n_items <= 0) return cudaSuccess;
    const BInst<T>* I = static_cast<const BInst<T>*>(L.inst);
    const int n = L.n_items;
    const dim3 cg(CL, n), pg(n), nt(cblk<T>()), vt(L.vec_nt), pt(L.pair_nt);
    const bool ph = L.pair_nt != cblk<T>(), t4 = L.taps == 4, v2 = L.vec_nt != PBLK;
    const T* const* pa = static_cast<const T* const*>(L.args);
    constexpr int NP = cblk<T>(), NH = cblk<T>() / 2;
    const ClArgs<T>* ca = static_cast<const ClArgs<T>*>(L.args);
    const SensorArgs<T>* sa = static_cast<const SensorArgs<T>*>(L.args);
    const VecArgs<T>* va = static_cast<const VecArgs<T>*>(L.args);
    const FitArgs<T>* fa = static_cast<const FitArgs<T>*>(L.args);
    switch (L.kind) {
        case BK_INV: return launch_b(L.pdl, kb_cl_inv<T, 0>, cg, nt, L.smem, st, I, ca, L.items);
        case BK_INV_UPD: return launch_b(L.pdl, kb_cl_inv<T, 1>, cg, nt, L.smem, st, I, ca, L.items);
        case BK_FWD_APPLY: return launch_b(L.pdl, kb_cl_fwd<T, LDST_APPLY>, cg, nt, L.smem, st, I, ca, L.items);
        case BK_FWD_COEF: return launch_b(L.pdl, kb_cl_fwd<T, LDST_COEF>, cg, nt, L.smem, st, I, ca, L.items);
        case BK_FWD_RINIT: return launch_b(L.pdl, kb_cl_fwd<T, LDST_RESID_INIT>, cg, nt, L.smem, st, I, ca, L.items);
        case BK_SEN_PHI: return launch_b(L.pdl, kb_cl_sensor<T, SSRC_PHI>, cg, nt, L.smem, st, I, sa, L.items);
        case BK_SEN_SLOPES: return launch_b(L.pdl, kb_cl_sensor<T, SSRC_SLOPES>, cg, nt, L.smem, st, I, sa, L.items);
        case BK_SEN_RESID: return launch_b(L.pdl, kb_cl_sensor<T, SSRC_RESID>, cg, nt, L.smem, st, I, sa, L.items);
        case BK_PROJ:
            return ph ? launch_b(L.pdl, kb_proj<T, NH>, pg, pt, L.smem, st, I, pa, L.items)
                      : launch_b(L.pdl, kb_proj<T, NP>, pg, pt, L.smem, st, I, pa, L.items);
        case BK_PROJT:
            if (t4)
                return ph ? launch_b(L.pdl, kb_projT<T, 4, NH>, pg, pt, L.smem, st, I, pa, L.items)
                          : launch_b(L.pdl, kb_projT<T, 4, NP>, pg, pt, L.smem, st, I, pa, L.items);
            return ph ? launch_b(L.pdl, kb_projT<T, KMAX, NH>, pg, pt, L.smem, st, I, pa, L.items)
                      : launch_b(L.pdl, kb_projT<T, KMAX, NP>, pg, pt, L.smem, st, I, pa, L.items);
        case BK_VEC_INIT:
            return v2 ? launch_b(L.pdl, kb_vec<T, V_INIT, 2 * PBLK>, pg, vt, 0, st, I, va, L.items)
                      : launch_b(L.pdl, kb_vec<T, V_INIT, PBLK>, pg, vt, 0, st, I, va, L.items);
        case BK_VEC_WARM:
            return v2 ? launch_b(L.pdl, kb_vec<T, V_INIT_WARM, 2 * PBLK>, pg, vt, 0, st, I, va, L.items)
                      : launch_b(L.pdl, kb_vec<T, V_INIT_WARM, PBLK>, pg, vt, 0, st, I, va, L.items);
        case BK_VEC_UPDATE:
            return v2 ? launch_b(L.pdl, kb_vec<T, V_UPDATE, 2 * PBLK>, pg, vt, 0, st, I, va, L.items)
                      : launch_b(L.pdl, kb_vec<T, V_UPDATE, PBLK>, pg, vt, 0, st, I, va, L.items);
        case BK_FIT: return launch_b(L.pdl, kb_fit<T>, pg, dim3(PBLK), L.smem, st, I, fa, L.items);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t batch_launch<float>(const BLaunch&, cudaStream_t);
template cudaError_t batch_launch<double>(const BLaunch&, cudaStream_t);
template cudaError_t batch_smem_limit<float>(int, size_t*);
template cudaError_t batch_smem_limit<double>(int, size_t*);

}  // namespace fewha
