// Persistent frame kernel: one cooperative launch of thread-block clusters runs a whole
// frame of Algorithm 1 (right-hand side, initial residual, the fixed PCG iterations of
// Sec. 3.3 and the DM fit), the stages separated by grid-wide barriers instead of kernel
// boundaries.  Every stage runs the same device bodies as the stream / graph form: a
// cluster per layer or sensor for the wavelet and sensor stages, the (sensor, layer) pairs
// spread over all CTAs for the projections, every CTA for the vector and fit stages.
//
// Every grid barrier waits a bounded number of polls.  A wait that runs out sets an abort
// flag (the other waits then give up at once) and an error bit the host maps to
// FEWHA_ERR_TIMEOUT, and the kernel returns: nothing waits forever.  The decision to go on
// or to return is taken by the leader of each cluster and broadcast to its CTAs through
// distributed shared memory before a cluster barrier, so the CTAs of a cluster always
// leave together and no cluster barrier is left waiting for an exited CTA.
#pragma once

#include "fewha_pair.cuh"

namespace fewha {

// Grid barrier state, in device memory; count and abort are zeroed before every launch.
struct GridSync {
    unsigned* count;     // arrivals, one per CTA and barrier (monotone within a launch)
    unsigned* abort;     // set by the first wait that runs out
    unsigned* status;    // bit 1 (value 2): a wait ran out
    unsigned limit;      // polls before a wait gives up
    unsigned extra;      // added to every target (tests: no wait can end)
    unsigned nctas;      // CTAs of the grid
};

// Barrier number k of the launch (k counted by the caller from 1).  Returns false, in every
// CTA of the cluster alike, when the frame is to stop.
__device__ __forceinline__ bool grid_barrier(const GridSync& gs, unsigned k) {
    __shared__ int gate;
    cg::cluster_group cluster = cg::this_cluster();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();                       // this CTA's writes before its arrival
        atomicAdd(gs.count, 1u);
    }
    if (cluster.block_rank() == 0 && threadIdx.x == 0) {
        const unsigned target = k * gs.nctas + gs.extra;
        int ok = 1;
        for (unsigned spins = 0;; ++spins) {
            if (ld_acquire_u32(gs.count) >= target) break;
            if (ld_acquire_u32(gs.abort) != 0u || spins >= gs.limit) {
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        if (!ok) {
            atomicOr(gs.abort, 1u);
            atomicOr(gs.status, 2u);
        }
        // every CTA of the cluster is running (they start together and all reach the
        // cluster barrier below), so the outcome can be pushed into their shared memory
        for (unsigned q = 0; q < cluster.num_blocks(); ++q) *cluster.map_shared_rank(&gate, q) = ok;
    }
    cluster.sync();
    const int ok = gate;
    if (threadIdx.x == 0) __threadfence();     // later loads see the other CTAs' writes
    __syncthreads();
    return ok != 0;
}

// Everything a persistent frame reads or writes.
template <class T>
struct FrameArgs {
    const T* s;          // slopes
    T* c;                // warm start, overwritten with the new iterate
    T* dm;               // commands
    T* a_prev;
    T* b;
    T* phi;
    T* u;
    T* q;
    VecArgs<T> v;        // r, z, p, b_prev, J^-1 and the PCG slots (npart = the grid's CTAs)
    unsigned* status;    // non-finite slopes (bit 0)
    int iters;
    int warm;            // r0 = (b - b_prev) + r_prev instead of b - M c0
    int apply_gain;      // 1: a = (1 - gain) a_prev + gain a~
    int pq_scratch;      // p.q slot of the initial-residual apply
};

// The stages as calls of their own (not inlined), so that each body is register-allocated
// alone rather than as one function with the whole frame.
template <class T, int PUPD>
__device__ __noinline__ void st_inv(const Desc<T>& d, const ClArgs<T>& a, const ClLayout& lay, int l) {
    cl_inv_body<T, PUPD>(d, a, lay, l);
}
template <class T, int SRC>
__device__ __noinline__ void st_sensor(const Desc<T>& d, const SensorArgs<T>& a, const SensorLayout& lay,
                                       const PairBufs<T>& pb, int g) {
    cl_sensor_body<T, SRC>(d, a, lay, pb, g);
}
template <class T, int DST>
__device__ __noinline__ void st_fwd(const Desc<T>& d, const ClArgs<T>& a, const ClLayout& lay, const PairBufs<T>& pb,
                                    int l, unsigned ctas) {
    cl_fwd_body<T, LSRC_NODES, DST>(d, a, lay, pb, l, ctas);
}
template <class T>
__device__ __noinline__ void st_proj(const Desc<T>& d, const T* phi, const PairBufs<T>& pb, int p0, int step) {
    for (int p = p0; p < d.n_layers * d.n_wfs; p += step) proj_body<T>(d, phi, pb, p / d.n_layers, p % d.n_layers);
}
template <class T>
__device__ __noinline__ void st_projT(const Desc<T>& d, const T* u, const PairBufs<T>& pb, int p0, int step) {
    for (int p = p0; p < d.n_layers * d.n_wfs; p += step) projT_body<T>(d, u, pb, p / d.n_layers, p % d.n_layers);
}
template <class T, int PHASE>
__device__ __noinline__ void st_vec(const Desc<T>& d, const VecArgs<T>& v, int cta, int nctas, int iter) {
    vec_body<T, PHASE, cblk<T>()>(d.n_c, v, cta, nctas, iter);
}
template <class T>
__device__ __noinline__ void st_fit(const Desc<T>& d, const T* phi, T* a_prev, T* dm, int gain, int cta, int nctas) {
    for (int blk = cta; blk * cblk<T>() < d.n_act; blk += nctas) fit_body<T, cblk<T>()>(d, phi, a_prev, dm, gain, blk);
}

template <class T>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(cblk<T>(), 1)
    k_frame(__grid_constant__ const Desc<T> d, __grid_constant__ const ClLayout lay_fwd,
            __grid_constant__ const ClLayout lay_inv, __grid_constant__ const SensorLayout lay_sen,
            __grid_constant__ const PairBufs<T> pb, __grid_constant__ const FrameArgs<T> f,
            __grid_constant__ const GridSync gs) {
    const int cl = blockIdx.y;                                   // cluster: a layer or a sensor
    const int cta = blockIdx.y * CL + blockIdx.x, nctas = gridDim.x * gridDim.y;
    const int nl = d.n_layers, nw = d.n_wfs;
    const unsigned lctas = static_cast<unsigned>(nl * CL);       // CTAs of a layer stage
    unsigned k = 0;
#define FEWHA_SYNC()                                 \
    do {                                             \
        if (!grid_barrier(gs, ++k)) return;          \
    } while (0)

    auto cl_args = [&](const T* in, T* out) {
        ClArgs<T> a{};
        a.in = in;
        a.out = out;
        a.pcg = f.v.pcg;
        return a;
    };
    // M x into qout (Eq. 6), the p.q partials into `slot`; pupd: x = p advanced first
    auto apply = [&](const T* x, T* qout, int slot, bool pupd) -> bool {
        if (cl < nl) {
            ClArgs<T> a = cl_args(x, f.phi);
            a.zero_piston = 1;
            if (pupd) {
                a.pupd = f.v.p;
                a.zupd = f.v.z;
                a.iter = slot;
                st_inv<T, 1>(d, a, lay_inv, cl);
            } else {
                st_inv<T, 0>(d, a, lay_inv, cl);
            }
        }
        if (!grid_barrier(gs, ++k)) return false;
        st_proj<T>(d, f.phi, pb, cta, nctas);
        if (!grid_barrier(gs, ++k)) return false;
        if (cl < nw) st_sensor<T, SSRC_PHI>(d, SensorArgs<T>{f.phi, f.u, f.status}, lay_sen, pb, cl);
        if (!grid_barrier(gs, ++k)) return false;
        st_projT<T>(d, f.u, pb, cta, nctas);
        if (!grid_barrier(gs, ++k)) return false;
        if (cl < nl) {
            ClArgs<T> a = cl_args(f.u, qout);
            a.pin = x;
            a.iter = slot;
            a.zero_piston = 1;
            st_fwd<T, LDST_APPLY>(d, a, lay_fwd, pb, cl, lctas);
        }
        return grid_barrier(gs, ++k);
    };

    // ---- right-hand side b = W sum_g P_g^T Gamma_g^T C_hat_g^-1 s_g (Sec. 3.1) ----------
    if (cl < nw) st_sensor<T, SSRC_SLOPES>(d, SensorArgs<T>{f.s, f.u, f.status}, lay_sen, pb, cl);
    FEWHA_SYNC();
    st_projT<T>(d, f.u, pb, cta, nctas);
    FEWHA_SYNC();
    if (cl < nl) {
        ClArgs<T> a = cl_args(f.u, f.b);
        a.zero_piston = 1;
        st_fwd<T, LDST_COEF>(d, a, lay_fwd, pb, cl, lctas);
    }
    FEWHA_SYNC();
    // ---- initial residual, explicit r0 = b - M c0 or the warm form -----------------------
    if (f.warm) {
        st_vec<T, V_INIT_WARM>(d, f.v, cta, nctas, 0);
    } else {
        if (!apply(f.c, f.q, f.pq_scratch, false)) return;
        st_vec<T, V_INIT>(d, f.v, cta, nctas, 0);
    }
    FEWHA_SYNC();
    // ---- PCG iterations (Sec. 3.3) --------------------------------------------------------
    for (int it = 0; it < f.iters; ++it) {
        if (!apply(f.v.p, f.q, it, it > 0)) return;
        st_vec<T, V_UPDATE>(d, f.v, cta, nctas, it);
        FEWHA_SYNC();
    }
    // ---- DM fit a~ = F W^T c and the control law (Algorithm 1) -----------------------------
    if (cl < nl) st_inv<T, 0>(d, cl_args(f.c, f.phi), lay_inv, cl);
    FEWHA_SYNC();
    st_fit<T>(d, f.phi, f.a_prev, f.dm, f.apply_gain, cta, nctas);
#undef FEWHA_SYNC
}

}  // namespace fewha
