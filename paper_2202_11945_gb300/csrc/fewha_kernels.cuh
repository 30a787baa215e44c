// sm_103a kernels of the FEWHA hot path.  No tensor cores: nothing here is a dense
// contraction; every kernel is a stencil, a gather or a reduction over data that
// stays in L2.  All reductions use a fixed thread-to-data map and fixed shuffle
// trees, and the adjoint operators are gathers (no atomics), so results are
// bitwise reproducible run to run.
#pragma once

#include <cuda_runtime.h>

#include "fewha_internal.h"

namespace fewha {

constexpr int BLK = 1024;   // threads of the per-layer and per-sensor kernels
constexpr int PQ_SLOTS = MAXL * 8;   // p.q partial slots per CG iteration (layer x cluster rank)
constexpr int PBLK = 256;   // threads of the vector (PCG) kernels

// Programmatic dependent launch: wait until the previous kernel has completed and its
// writes are visible, then let the stream's next kernel start launching its CTAs.  Both
// instructions are no-ops when the kernel was launched without programmatic stream
// serialization.
//
// Every kernel lets the next one launch only after its own wait.  So while any CTA of a
// kernel runs, the kernel two places before it in the stream has completed, and a kernel
// may read, before its wait, data that no kernel closer than that wrote (the forward layer
// kernel prefetches its epilogue operands this way).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}
// The cluster kernels trigger later, from a barrier in their middle: launched at their
// entry, the next kernel's CTAs would take SMs and issue slots for most of the long
// cluster kernel (measured slower on GB300); launched from the middle, they are resident
// and waiting when it ends.
constexpr int NWARP = BLK / 32;

__constant__ float c_h32[6];
__constant__ float c_g32[6];
__constant__ double c_h64[6];
__constant__ double c_g64[6];

template <class T> __device__ __forceinline__ T tap_h(int t);
template <class T> __device__ __forceinline__ T tap_g(int t);
template <> __device__ __forceinline__ float tap_h<float>(int t) { return c_h32[t]; }
template <> __device__ __forceinline__ float tap_g<float>(int t) { return c_g32[t]; }
template <> __device__ __forceinline__ double tap_h<double>(int t) { return c_h64[t]; }
template <> __device__ __forceinline__ double tap_g<double>(int t) { return c_g64[t]; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Inner products of the PCG (Sec. 3.3) to double accuracy.  In the FP32 form a thread's
// share is accumulated in double-float (compensated FP32) arithmetic: the product of two
// floats is exact as hi + lo (hi = fl(p q), lo = fma(p, q, -hi)), and the running sum is
// an unevaluated s + c updated by a two-sum per term (relative error about 2^-48).  This
// runs on the FP32 pipes; GB300's FP64 rate is about 1/64 of its FP32 rate, so converting
// and accumulating every product in FP64 dominated the epilogues that form p.q and r.z.
// The _rn intrinsics keep the compiler from fusing the two-sum steps.  A CTA's shares are
// merged in the same arithmetic in a fixed order and leave the CTA as one double; totals
// over CTAs, and alpha and beta, stay in FP64.  The FP64 form accumulates in double.
// ---------------------------------------------------------------------------
struct DFloat {
    float s, c;    // value s + c, |c| small against |s|
};

__device__ __forceinline__ DFloat df_merge(DFloat a, DFloat b) {
    const float t = __fadd_rn(a.s, b.s);                     // two-sum of the leading parts
    const float bp = __fsub_rn(t, a.s);
    const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(b.s, bp));
    const float c = __fadd_rn(__fadd_rn(a.c, b.c), e);
    const float s = __fadd_rn(t, c);                         // renormalise (fast two-sum)
    return DFloat{s, __fsub_rn(c, __fsub_rn(s, t))};
}

template <class T>
struct DotAcc;

template <>
struct DotAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double p, double q) { v += p * q; }
};

template <>
struct DotAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float p, float q) {
        const float h = __fmul_rn(p, q);
        const float l = __fmaf_rn(p, q, -h);                 // p q = h + l exactly
        const float t = __fadd_rn(s, h);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(h, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(e, l));
    }
};

// Fixed-order CTA total of the threads' shares, returned to every thread.  `scratch`
// holds blockDim.x doubles.
__device__ __forceinline__ double cta_dot(const DotAcc<double>& a, double* scratch) {
    const int nt = blockDim.x;
    scratch[threadIdx.x] = a.v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = 0.0;
        for (int i = threadIdx.x; i < nt; i += 32) x += scratch[i];
        x = warp_sum(x);
        if (threadIdx.x == 0) scratch[0] = x;
    }
    __syncthreads();
    const double r = scratch[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ DFloat warp_df_sum(DFloat v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const DFloat w{__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)};
        v = df_merge(v, w);
    }
    return v;
}

__device__ __forceinline__ double cta_dot(const DotAcc<float>& a, double* scratch) {
    float2* sh = reinterpret_cast<float2*>(scratch);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const DFloat v = warp_df_sum(DFloat{a.s, a.c});
    if (lane == 0) sh[warp] = make_float2(v.s, v.c);
    __syncthreads();
    if (warp == 0) {
        const float2 x = lane < nw ? sh[lane] : make_float2(0.f, 0.f);
        const DFloat t = warp_df_sum(DFloat{x.x, x.y});
        if (lane == 0) scratch[0] = double(t.s) + double(t.c);
    }
    __syncthreads();
    const double r = scratch[0];
    __syncthreads();
    return r;
}

// A CTA's share of an inner product into its 8-byte slot, for the last-arriving CTA to
// total (fixed order).  The FP64 form stores the double; the FP32 form stores the
// double-float pair (s, c) itself, so that the total is also formed on the FP32 pipes.
// The slot is written by thread 0 (last_arrival orders it before the arrival count).
__device__ __forceinline__ void cta_dot_store(const DotAcc<double>& a, double* scratch, double* slot) {
    const double x = cta_dot(a, scratch);
    if (threadIdx.x == 0) *slot = x;
}

__device__ __forceinline__ void cta_dot_store(const DotAcc<float>& a, double* scratch, double* slot) {
    float2* sh = reinterpret_cast<float2*>(scratch);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const DFloat v = warp_df_sum(DFloat{a.s, a.c});
    if (lane == 0) sh[warp] = make_float2(v.s, v.c);
    __syncthreads();
    if (warp == 0) {
        const float2 x = lane < nw ? sh[lane] : make_float2(0.f, 0.f);
        const DFloat t = warp_df_sum(DFloat{x.x, x.y});
        if (lane == 0) *reinterpret_cast<float2*>(slot) = make_float2(t.s, t.c);
    }
}

// Total of `cnt` <= 512 slots written by other CTAs, by one warp in a fixed order: every
// lane issues its loads at once (L2, bypassing L1), then a fixed tree.  Valid in lane 0.
__device__ __forceinline__ double warp_total(const double* p, int cnt, const DotAcc<double>*) {
    double v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int i = (threadIdx.x & 31) + 32 * k;
        v[k] = i < cnt ? __ldcg(p + i) : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += v[k];
    return warp_sum(s);
}

__device__ __forceinline__ double warp_total(const double* p, int cnt, const DotAcc<float>*) {
    float2 v[16];
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int i = (threadIdx.x & 31) + 32 * k;
        v[k] = i < cnt ? __ldcg(q + i) : make_float2(0.f, 0.f);
    }
    DFloat s{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 16; ++k) s = df_merge(s, DFloat{v[k].x, v[k].y});
    s = warp_df_sum(s);
    return double(s.s) + double(s.c);
}

// LGS spot elongation of subaperture (i, j) (Eq. 3): beta and gamma, so that
// C_ij^-1 = sigma^-2 (I - gamma beta beta^T) (Sherman-Morrison).
__device__ __forceinline__ void elong(const WfsInfo& W, int i, int j, double& b1, double& b2, double& gam) {
    b1 = W.el_k * ((W.el_x0 + j * W.el_d) - W.el_lx);
    b2 = W.el_k * ((W.el_x0 + i * W.el_d) - W.el_ly);
    gam = W.el_c / (1.0 + W.el_c * (b1 * b1 + b2 * b2));
}
__device__ __forceinline__ void elong(const WfsInfo& W, int i, int j, float& b1, float& b2, float& gam) {
    b1 = W.el_f[0] * ((W.el_f[4] + float(j) * W.el_f[5]) - W.el_f[2]);
    b2 = W.el_f[0] * ((W.el_f[4] + float(i) * W.el_f[5]) - W.el_f[3]);
    gam = W.el_f[1] / (1.f + W.el_f[1] * (b1 * b1 + b2 * b2));
}
// K11, K12, K22 (q = 0, 1, 2) of the sensor in the kernel's precision.
__device__ __forceinline__ double el_K(const WfsInfo& W, int q, double) {
    return q == 0 ? W.el_K11 : (q == 1 ? W.el_K12 : W.el_K22);
}
__device__ __forceinline__ float el_K(const WfsInfo& W, int q, float) { return W.el_f[6 + q]; }

// Deterministic block sum of two doubles (fixed tree); red holds >= 2*(NWARP+1).
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    if (lane == 0) {
        red[w] = a;
        red[NWARP + w] = b;
    }
    __syncthreads();
    if (w == 0) {
        double x = lane < nw ? red[lane] : 0.0;
        double y = lane < nw ? red[NWARP + lane] : 0.0;
        x = warp_sum(x);
        y = warp_sum(y);
        if (lane == 0) {
            red[2 * NWARP] = x;
            red[2 * NWARP + 1] = y;
        }
    }
    __syncthreads();
    a = red[2 * NWARP];
    b = red[2 * NWARP + 1];
    __syncthreads();
}

// Sum of cnt doubles in a fixed order, computed by warp 0 and broadcast via *out.
__device__ __forceinline__ double sum_partials(const double* p, int cnt, double* slot) {
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = threadIdx.x; i < cnt; i += 32) v += p[i];
        v = warp_sum(v);
        if (threadIdx.x == 0) *slot = v;
    }
    __syncthreads();
    const double r = *slot;
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Periodic Daubechies-3 steps on the m x m top-left block of an n x n shared tile.
// Analysis: a_k = sum_t h_t x_(2k+t mod m), d_k = sum_t g_t x_(2k+t mod m) (Sec. 3.1).
// Each thread owns (a_k, d_k) pairs; results go through registers so the step is
// in place.  m*m/2 <= 8192 pairs = 8 per thread at n = 128.
// ---------------------------------------------------------------------------
constexpr int PAIRS = (MAXN * MAXN / 2 + BLK - 1) / BLK;

template <class T>
__device__ __forceinline__ void fwd_rows(T* S, int n, int m, int lm) {
    const int h = m >> 1, lh = lm - 1, pairs = m * h;
    T ra[PAIRS], rd[PAIRS];
#pragma unroll
    for (int it = 0; it < PAIRS; ++it) {
        const int idx = threadIdx.x + it * BLK;
        if (idx < pairs) {
            const int r = idx >> lh, k = idx & (h - 1);
            const T* row = S + r * n;
            T a = T(0), d = T(0);
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                const T x = row[(2 * k + t) & (m - 1)];
                a += tap_h<T>(t) * x;
                d += tap_g<T>(t) * x;
            }
            ra[it] = a;
            rd[it] = d;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < PAIRS; ++it) {
        const int idx = threadIdx.x + it * BLK;
        if (idx < pairs) {
            const int r = idx >> lh, k = idx & (h - 1);
            S[r * n + k] = ra[it];
            S[r * n + h + k] = rd[it];
        }
    }
    __syncthreads();
}

template <class T>
__device__ __forceinline__ void fwd_cols(T* S, int n, int m, int lm) {
    const int h = m >> 1, pairs = m * h;
    T ra[PAIRS], rd[PAIRS];
#pragma unroll
    for (int it = 0; it < PAIRS; ++it) {
        const int idx = threadIdx.x + it * BLK;
        if (idx < pairs) {
            const int c = idx & (m - 1), k = idx >> lm;
            T a = T(0), d = T(0);
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                const T x = S[((2 * k + t) & (m - 1)) * n + c];
                a += tap_h<T>(t) * x;
                d += tap_g<T>(t) * x;
            }
            ra[it] = a;
            rd[it] = d;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < PAIRS; ++it) {
        const int idx = threadIdx.x + it * BLK;
        if (idx < pairs) {
            const int c = idx & (m - 1), k = idx >> lm;
            S[k * n + c] = ra[it];
            S[(h + k) * n + c] = rd[it];
        }
    }
    __syncthreads();
}

// Synthesis (transpose of the analysis): outputs 2k and 2k+1 take a_k, a_(k-1),
// a_(k-2) and the same d's (indices mod m/2):
//   x_2k   = h0 a_k + h2 a_(k-1) + h4 a_(k-2) + g0 d_k + g2 d_(k-1) + g4 d_(k-2)
//   x_2k+1 = h1 a_k + h3 a_(k-1) + h5 a_(k-2) + g1 d_k + g3 d_(k-1) + g5 d_(k-2)
template <class T>
__device__ __forceinline__ void inv_cols(T* S, int n, int m, int lm) {
    const int h = m >> 1, pairs = m * h;
    T re[PAIRS], ro[PAIRS];
#pragma unroll
    for (int it = 0; it < PAIRS; ++it) {
        const int idx = threadIdx.x + it * BLK;
        if (idx < pairs) {
            const int c = idx & (m - 1), k = idx >> lm;
            const int k1 = (k - 1) & (h - 1), k2 = (k - 2) & (h - 1);
            const T a0 = S[k * n + c], a1 = S[k1 * n + c], a2 = S[k2 * n + c];
            const T d0 = S[(h + k) * n + c], d1 = S[(h + k1) * n + c], d2 = S[(h + k2) * n + c];
            re[it] = tap_h<T>(0) * a0 + tap_h<T>(2) * a1 + tap_h<T>(4) * a2 +
                     tap_g<T>(0) * d0 + tap_g<T>(2) * d1 + tap_g<T>(4) * d2;
            ro[it] = tap_h<T>(1) * a0 + tap_h<T>(3) * a1 + tap_h<T>(5) * a2 +
                     tap_g<T>(1) * d0 + tap_g<T>(3) * d1 + tap_g<T>(5) * d2;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < PAIRS; ++it) {
        const int idx = threadIdx.x + it * BLK;
        if (idx < pairs) {
            const int c = idx & (m - 1), k = idx >> lm;
            S[(2 * k) * n + c] = re[it];
            S[(2 * k + 1) * n + c] = ro[it];
        }
    }
    __syncthreads();
}

template <class T>
__device__ __forceinline__ void inv_rows(T* S, int n, int m, int lm) {
    const int h = m >> 1, lh = lm - 1, pairs = m * h;
    T re[PAIRS], ro[PAIRS];
#pragma unroll
    for (int it = 0; it < PAIRS; ++it) {
        const int idx = threadIdx.x + it * BLK;
        if (idx < pairs) {
            const int r = idx >> lh, k = idx & (h - 1);
            const int k1 = (k - 1) & (h - 1), k2 = (k - 2) & (h - 1);
            const T* row = S + r * n;
            const T a0 = row[k], a1 = row[k1], a2 = row[k2];
            const T d0 = row[h + k], d1 = row[h + k1], d2 = row[h + k2];
            re[it] = tap_h<T>(0) * a0 + tap_h<T>(2) * a1 + tap_h<T>(4) * a2 +
                     tap_g<T>(0) * d0 + tap_g<T>(2) * d1 + tap_g<T>(4) * d2;
            ro[it] = tap_h<T>(1) * a0 + tap_h<T>(3) * a1 + tap_h<T>(5) * a2 +
                     tap_g<T>(1) * d0 + tap_g<T>(3) * d1 + tap_g<T>(5) * d2;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < PAIRS; ++it) {
        const int idx = threadIdx.x + it * BLK;
        if (idx < pairs) {
            const int r = idx >> lh, k = idx & (h - 1);
            S[r * n + 2 * k] = re[it];
            S[r * n + 2 * k + 1] = ro[it];
        }
    }
    __syncthreads();
}

template <class T>
__device__ __forceinline__ void dwt_forward(T* S, const LayerInfo& L) {
    for (int lev = 0; lev < L.levels; ++lev) {
        const int m = L.n >> lev, lm = L.log2n - lev;
        fwd_rows(S, L.n, m, lm);
        fwd_cols(S, L.n, m, lm);
    }
}

template <class T>
__device__ __forceinline__ void dwt_inverse(T* S, const LayerInfo& L) {
    for (int lev = L.levels - 1; lev >= 0; --lev) {
        const int m = L.n >> lev, lm = L.log2n - lev;
        inv_cols(S, L.n, m, lm);
        inv_rows(S, L.n, m, lm);
    }
}

// Level of position (i, j) of a layer in Mallat layout: detail level k (1 = finest) where
// n / 2^k <= max(i, j) < n / 2^(k-1), and levels + 1 for the LL band.
__device__ __forceinline__ int level_of(int i, int j, const LayerInfo& L) {
    const int m = max(i, j);
    return m < (L.n >> L.levels) ? L.levels + 1 : L.log2n - (31 - __clz(m));
}

// ---------------------------------------------------------------------------
// PCG bookkeeping: per-iteration partial inner products in fixed slots.
// rz of iteration k = sum of rzpart[k * npart + 0 .. npart); p.q of iteration k =
// sum of pqpart[k * MAXL + 0 .. n_layers).
// ---------------------------------------------------------------------------
struct PcgSlots {
    double* rzpart;     // [slot * npart + cta]: partial r.z
    double* pqpart;     // [slot * PQ_SLOTS + l * 8 + rank]: partial p.q
    double* rztot;      // [slot]: r.z in fixed summation order (slot 0: initial residual)
    double* pqtot;      // [slot]: p.q of iteration slot
    unsigned* count;    // [2]: arrival counters of the reducing grids, reset by the last CTA
    int npart;
};

// Arrival of one CTA of a reducing grid; true in the CTA that arrives last.  Its
// partial must already be stored; the fence orders it before the count.
__device__ __forceinline__ bool last_arrival(unsigned* count, unsigned ctas, bool* flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(count, 1u);
        *flag = (prev == ctas - 1);
    }
    __syncthreads();
    const bool last = *flag;
    if (last) __threadfence();
    return last;
}

// ---------------------------------------------------------------------------
// Per-layer kernel.  Source: the layer values (SRC_PHI), the adjoint projection of
// aperture-node vectors (SRC_NODES, P^T as a gather), or the adjoint DM fit
// (SRC_DM).  Destination: layer values (DST_PHI), wavelet coefficients (DST_COEF),
// or q = W y + alpha D p with the partial p.q (DST_APPLY).
// PUPDATE: before use, the CG direction of this layer is advanced, p = z + beta p,
// beta = rz_k / rz_(k-1) (Sec. 3.3; the update is fused into the first kernel of
// iteration k).
// ---------------------------------------------------------------------------
enum { LSRC_PHI = 0, LSRC_NODES = 1, LSRC_DM = 2, LSRC_COEF = 3 };
// LDST_APPLY_INIT: the forward cluster kernel's apply with the initial residual's vector
// step fused into its epilogue
// LDST_RESID_INIT: the same vector step with the data term already the residual's (the
// sensor kernel's SSRC_RESID): r0 = W y - alpha D c0, with no b
enum { LDST_PHI = 0, LDST_COEF = 1, LDST_APPLY = 2, LDST_APPLY_INIT = 3, LDST_RESID_INIT = 4 };

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <class T>
struct LayerArgs {
    const T* in;      // source vector
    const T* pin;     // p of the apply (DST_APPLY)
    T* out;           // destination vector
    T* pupd;          // p to advance (PUPDATE), updated in place
    const T* zupd;    // z of the update
    PcgSlots pcg;
    int iter;         // CG iteration of the apply / update
    int zero_piston;  // data term: the full-depth LL coefficient is exactly 0
};

template <class T, int SRC, int DST, bool PUPDATE>
__global__ void __launch_bounds__(BLK) k_layer(const Desc<T> d, const LayerArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);          // 2*NWARP + 4 doubles
    T* S = reinterpret_cast<T*>(red + 2 * NWARP + 4);
    const int l = blockIdx.x;
    const LayerInfo L = d.L[l];
    const int n = L.n, nn = n * n, off = L.off;

    if (PUPDATE) {
        const double rz_new = sum_partials(a.pcg.rzpart + a.iter * a.pcg.npart, a.pcg.npart, red);
        const double rz_old = sum_partials(a.pcg.rzpart + (a.iter - 1) * a.pcg.npart, a.pcg.npart, red);
        const T beta = rz_old != 0.0 ? T(rz_new / rz_old) : T(0);
        for (int k = threadIdx.x; k < nn; k += BLK) {
            const T p = a.zupd[off + k] + beta * a.pupd[off + k];
            a.pupd[off + k] = p;
            S[k] = p;
        }
    } else if (SRC == LSRC_PHI || SRC == LSRC_COEF) {
        for (int k = threadIdx.x; k < nn; k += BLK) S[k] = a.in[off + k];
    } else if (SRC == LSRC_NODES) {
        // y(i, j) = sum_g sum_a sum_b wy(a, i) wx(b, j) u_g(a, b): P_g^T as a gather over
        // the aperture nodes whose bilinear stencil touches layer node (i, j).
        for (int k = threadIdx.x; k < nn; k += BLK) {
            const int i = k >> L.log2n, j = k & (n - 1);
            T acc = T(0);
            for (int g = 0; g < d.n_wfs; ++g) {
                const int rb = (g * MAXL + l) * MAXN;
                const int a0 = d.ry_lo[rb + i], a1 = d.ry_hi[rb + i];
                const int b0 = d.rx_lo[rb + j], b1 = d.rx_hi[rb + j];
                if (a0 >= a1 || b0 >= b1) continue;
                const int tp = (g * MAXL + l) * TAB;
                const int NP = d.G[g].N + 1;
                const T* u = a.in + d.G[g].node_off;
                for (int aa = a0; aa < a1; ++aa) {
                    const T wy = d.pi0y[tp + aa] == i ? T(1) - d.pfy[tp + aa] : d.pfy[tp + aa];
                    T row = T(0);
                    for (int bb = b0; bb < b1; ++bb) {
                        const T wx = d.pi0x[tp + bb] == j ? T(1) - d.pfx[tp + bb] : d.pfx[tp + bb];
                        row += wx * u[aa * NP + bb];
                    }
                    acc += wy * row;
                }
            }
            S[k] = acc;
        }
    } else if (SRC == LSRC_DM) {
        // adjoint of the DM fit: y(i, j) = sum_m w_lm sum_p sum_q wy(p, i) wx(q, j) a_m(p, q)
        for (int k = threadIdx.x; k < nn; k += BLK) {
            const int i = k >> L.log2n, j = k & (n - 1);
            T acc = T(0);
            for (int m = 0; m < d.n_dms; ++m) {
                const T w = d.fitw[m][l];
                if (w == T(0)) continue;
                const int rb = (m * MAXL + l) * MAXN;
                const int p0 = d.dr_lo[rb + i], p1 = d.dr_hi[rb + i];
                const int q0 = d.dr_lo[rb + j], q1 = d.dr_hi[rb + j];
                if (p0 >= p1 || q0 >= q1) continue;
                const int tb = (m * MAXL + l) * MAXNACT;
                const int na = d.Mi[m].n_act;
                const T* am = a.in + d.Mi[m].off;
                T sm = T(0);
                for (int p = p0; p < p1; ++p) {
                    const T wy = d.di0[tb + p] == i ? T(1) - d.dfw[tb + p] : d.dfw[tb + p];
                    T row = T(0);
                    for (int q = q0; q < q1; ++q) {
                        const T wx = d.di0[tb + q] == j ? T(1) - d.dfw[tb + q] : d.dfw[tb + q];
                        row += wx * am[p * na + q];
                    }
                    sm += wy * row;
                }
                acc += w * sm;
            }
            S[k] = acc;
        }
    }
    __syncthreads();

    if (DST == LDST_PHI) {
        if (SRC == LSRC_COEF || PUPDATE) dwt_inverse(S, L);
        for (int k = threadIdx.x; k < nn; k += BLK) a.out[off + k] = S[k];
        return;
    }
    dwt_forward(S, L);
    // The data term has no piston component: Gamma annihilates constants and bilinear
    // weights sum to one, so (W P^T Gamma^T ...)_LL = 0 exactly at full depth.  Write
    // that zero instead of the rounding residue of a cancelling sum (it would be
    // amplified by 1 / (alpha D_LL) in the solve).
    if (a.zero_piston && L.full && threadIdx.x == 0) S[0] = T(0);
    __syncthreads();
    if (DST == LDST_COEF) {
        for (int k = threadIdx.x; k < nn; k += BLK) a.out[off + k] = S[k];
        return;
    }
    // DST_APPLY: q = W B W^T p + alpha D p, partial p.q in double
    double dot = 0.0, dummy = 0.0;
    for (int k = threadIdx.x; k < nn; k += BLK) {
        const T p = a.pin[off + k];
        const T q = S[k] + d.alpha * d.D[off + k] * p;
        a.out[off + k] = q;
        dot += double(p) * double(q);
    }
    block_sum2(dot, dummy, red);
    if (threadIdx.x == 0) a.pcg.pqpart[a.iter * MAXL + l] = dot;
}

// ---------------------------------------------------------------------------
// Per-sensor kernel (one CTA per sensor): projection P_g, Shack-Hartmann slopes
// Gamma_g, noise weighting C_hat_g^-1 (Eq. 2, Sec. 3.2) and Gamma_g^T, selected by
// SRC / WEIGHT / DST.  Shared tiles: V (aperture nodes), SX, SY (per subaperture,
// zero outside the active set).
// ---------------------------------------------------------------------------
// SSRC_RESID (cluster sensor kernel only): the measured slopes (in) minus the projected
// layers' slopes, the initial residual's data term before the noise weighting
enum { SSRC_PHI = 0, SSRC_NODES = 1, SSRC_SLOPES = 2, SSRC_RESID = 3 };
enum { SDST_NODES = 0, SDST_SLOPES = 1, SDST_ADJ = 2 };

template <class T>
struct SensorArgs {
    const T* in;
    T* out;
    unsigned* status;   // bit 0: a non-finite input slope was seen
};

template <class T, int SRC, bool WEIGHT, int DST>
__global__ void __launch_bounds__(BLK) k_sensor(const Desc<T> d, const SensorArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);          // 2*NWARP + 4
    double* csum = red + 2 * NWARP + 4;                          // 2*MAXCOARSE
    const int g = blockIdx.x;
    const WfsInfo W = d.G[g];
    const int N = W.N, NP = N + 1, NN = N * N, NPP = NP * NP;
    T* V = reinterpret_cast<T*>(csum + 2 * MAXCOARSE);
    T* SX = V + NPP;
    T* SY = SX + NN;
    const int* sidx = d.sidx + W.mask_off;
    const T inv = T(W.sig2inv);
    const T nbinv = T(1) / T(W.nb);

    // ---- source -----------------------------------------------------------
    if (SRC == SSRC_PHI) {
        // P_g (Sec. 2): phi_g(x) = sum_l phi_l(s_l x + theta h_l), bilinear
        for (int k = threadIdx.x; k < NPP; k += BLK) {
            const int aa = k / NP, bb = k - aa * NP;
            T v = T(0);
            for (int l = 0; l < d.n_layers; ++l) {
                const int tp = (g * MAXL + l) * TAB;
                const int i0 = d.pi0y[tp + aa], j0 = d.pi0x[tp + bb];
                const T fy = d.pfy[tp + aa], fx = d.pfx[tp + bb];
                const int n = d.L[l].n;
                const T* P = a.in + d.L[l].off + i0 * n + j0;
                v += (T(1) - fy) * ((T(1) - fx) * P[0] + fx * P[1]) +
                     fy * ((T(1) - fx) * P[n] + fx * P[n + 1]);
            }
            V[k] = v;
        }
    } else if (SRC == SSRC_NODES) {
        for (int k = threadIdx.x; k < NPP; k += BLK) V[k] = a.in[W.node_off + k];
    } else {
        // measured slopes -> per-subaperture tiles (coarse: spread over the block, 1/nb)
        const T* s = a.in + W.soff;
        bool bad = false;
        for (int k = threadIdx.x; k < NN; k += BLK) {
            const int id = sidx[k];
            T sx = T(0), sy = T(0);
            if (id >= 0) {
                sx = s[id];
                sy = s[W.n_active + id];
                bad |= !(isfinite(sx) && isfinite(sy));
                if (W.nb > 1) {
                    sx *= nbinv;
                    sy *= nbinv;
                    if (WEIGHT) {
                        sx *= inv;
                        sy *= inv;
                    }
                }
            }
            SX[k] = sx;
            SY[k] = sy;
        }
        if (bad && a.status) atomicOr(a.status, 1u);
    }
    __syncthreads();
    if (SRC != SSRC_SLOPES && DST == SDST_NODES) {
        for (int k = threadIdx.x; k < NPP; k += BLK) a.out[W.node_off + k] = V[k];
        return;
    }

    // ---- Gamma_g: slopes of the active fine subapertures (Sec. 2, y-slope read as
    // the mirror of the x-slope) ----------------------------------------------------
    if (SRC != SSRC_SLOPES) {
        for (int k = threadIdx.x; k < NN; k += BLK) {
            const int i = k / N, j = k - i * N;
            T sx = T(0), sy = T(0);
            if (sidx[k] >= 0) {
                const T v00 = V[i * NP + j], v01 = V[i * NP + j + 1];
                const T v10 = V[(i + 1) * NP + j], v11 = V[(i + 1) * NP + j + 1];
                sx = T(0.5) * ((v01 - v00) + (v11 - v10));
                sy = T(0.5) * ((v10 - v00) + (v11 - v01));
            }
            SX[k] = sx;
            SY[k] = sy;
        }
        __syncthreads();
        if (W.nb > 1) {
            // coarse sensor: slope_K = (1/nb) sum of the active fine slopes in block K
            const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
            const int ns = W.n_sub, nb = W.nb;
            for (int blk = w; blk < ns * ns; blk += NWARP) {
                const int K = d.cidx[W.cmask_off + blk];
                if (K < 0) continue;
                const int I = blk / ns, J = blk - I * ns;
                double sx = 0.0, sy = 0.0;
                for (int t = lane; t < nb * nb; t += 32) {
                    const int r = t / nb, c = t - r * nb;
                    const int k = (I * nb + r) * N + J * nb + c;
                    sx += double(SX[k]);
                    sy += double(SY[k]);
                }
                sx = warp_sum(sx);
                sy = warp_sum(sy);
                if (lane == 0) {
                    csum[2 * K] = sx / nb;
                    csum[2 * K + 1] = sy / nb;
                }
            }
            __syncthreads();
            if (DST == SDST_SLOPES) {
                for (int K = threadIdx.x; K < W.n_active; K += BLK) {
                    T cx = T(csum[2 * K]), cy = T(csum[2 * K + 1]);
                    if (WEIGHT) {
                        cx *= inv;
                        cy *= inv;
                    }
                    a.out[W.soff + K] = cx;
                    a.out[W.soff + W.n_active + K] = cy;
                }
                return;
            }
            // spread the (weighted) coarse slopes back over the fine subapertures:
            // Gamma_coarse^T puts slope_K / nb on every active fine subaperture of K
            for (int k = threadIdx.x; k < NN; k += BLK) {
                const int id = sidx[k];
                T sx = T(0), sy = T(0);
                if (id >= 0) {
                    sx = T(csum[2 * id]) * nbinv;
                    sy = T(csum[2 * id + 1]) * nbinv;
                    if (WEIGHT) {
                        sx *= inv;
                        sy *= inv;
                    }
                }
                SX[k] = sx;
                SY[k] = sy;
            }
            __syncthreads();
        }
    }

    // ---- C_hat_g^-1 on fine sensors: LGS (I - T) sigma^-2 (I - T) = sigma^-2 (I - T),
    // T removing the mean x- and y-slope over the active set (Sec. 3.2); NGS sigma^-2.
    if (WEIGHT && W.nb == 1) {
        if (W.lgs) {
            double tx = 0.0, ty = 0.0, ex = 0.0, ey = 0.0;
            for (int k = threadIdx.x; k < NN; k += BLK) {
                tx += double(SX[k]);
                ty += double(SY[k]);
                if (W.el && sidx[k] >= 0) {
                    T b1, b2, gam;
                    elong(W, k / N, k % N, b1, b2, gam);
                    const T bs = b1 * SX[k] + b2 * SY[k];
                    ex += double(gam * b1 * bs);
                    ey += double(gam * b2 * bs);
                }
            }
            block_sum2(tx, ty, red);
            if (W.el) block_sum2(ex, ey, red);
            const T mx = T(tx / W.n_active), my = T(ty / W.n_active);
            // elongated: C_hat^-1 s = sigma^-2 (u - gamma beta (beta . u) + g), u = s minus
            // its means, g = (e - K m) / |M| the mean of gamma beta (beta . u)
            const T g1 = T((ex - (W.el_K11 * double(mx) + W.el_K12 * double(my))) / W.n_active);
            const T g2 = T((ey - (W.el_K12 * double(mx) + W.el_K22 * double(my))) / W.n_active);
            for (int k = threadIdx.x; k < NN; k += BLK) {
                if (sidx[k] >= 0) {
                    const T ux = SX[k] - mx, uy = SY[k] - my;
                    if (W.el) {
                        T b1, b2, gam;
                        elong(W, k / N, k % N, b1, b2, gam);
                        const T bu = b1 * ux + b2 * uy;
                        SX[k] = inv * ((ux - gam * b1 * bu) + g1);
                        SY[k] = inv * ((uy - gam * b2 * bu) + g2);
                    } else {
                        SX[k] = inv * ux;
                        SY[k] = inv * uy;
                    }
                }
            }
        } else {
            for (int k = threadIdx.x; k < NN; k += BLK) {
                SX[k] *= inv;
                SY[k] *= inv;
            }
        }
        __syncthreads();
    }

    // ---- destination ------------------------------------------------------------
    if (DST == SDST_SLOPES) {
        if (W.nb > 1) {
            // slopes in -> (weighted) slopes out on a coarse sensor
            for (int K = threadIdx.x; K < W.n_active; K += BLK) {
                T cx = a.in[W.soff + K], cy = a.in[W.soff + W.n_active + K];
                if (WEIGHT) {
                    cx *= inv;
                    cy *= inv;
                }
                a.out[W.soff + K] = cx;
                a.out[W.soff + W.n_active + K] = cy;
            }
            return;
        }
        for (int k = threadIdx.x; k < NN; k += BLK) {
            const int id = sidx[k];
            if (id >= 0) {
                a.out[W.soff + id] = SX[k];
                a.out[W.soff + W.n_active + id] = SY[k];
            }
        }
        return;
    }
    // Gamma_g^T: u(a, b) = 1/2 [sx(a, b-1) - sx(a, b) + sx(a-1, b-1) - sx(a-1, b)]
    //                    + 1/2 [sy(a-1, b) - sy(a, b) + sy(a-1, b-1) - sy(a, b-1)]
    for (int k = threadIdx.x; k < NPP; k += BLK) {
        const int aa = k / NP, bb = k - aa * NP;
        const bool r0 = aa < N, r1 = aa > 0, c0 = bb < N, c1 = bb > 0;
        const T x_ab = (r0 && c0) ? SX[aa * N + bb] : T(0);
        const T x_ab1 = (r0 && c1) ? SX[aa * N + bb - 1] : T(0);
        const T x_a1b = (r1 && c0) ? SX[(aa - 1) * N + bb] : T(0);
        const T x_a1b1 = (r1 && c1) ? SX[(aa - 1) * N + bb - 1] : T(0);
        const T y_ab = (r0 && c0) ? SY[aa * N + bb] : T(0);
        const T y_ab1 = (r0 && c1) ? SY[aa * N + bb - 1] : T(0);
        const T y_a1b = (r1 && c0) ? SY[(aa - 1) * N + bb] : T(0);
        const T y_a1b1 = (r1 && c1) ? SY[(aa - 1) * N + bb - 1] : T(0);
        a.out[W.node_off + k] =
            T(0.5) * ((x_ab1 - x_ab) + (x_a1b1 - x_a1b)) + T(0.5) * ((y_a1b - y_ab) + (y_a1b1 - y_ab1));
    }
}

// ---------------------------------------------------------------------------
// PCG vector kernels (Sec. 3.3, standard left-preconditioned CG).  Vectors in T,
// inner products and the scalars alpha = rz/pq, beta = rz_new/rz in double.
// ---------------------------------------------------------------------------
template <class T>
struct VecArgs {
    T* c;
    T* r;
    T* z;
    T* p;
    const T* q;
    const T* b;
    T* b_prev;
    const T* Jinv;
    PcgSlots pcg;
    int iter;
    // V_UPDATE with deferred totals: pq_cnt > 0, the p.q total of the iteration is formed
    // here from the forward kernel's pq_cnt shares (fixed order) and stored by CTA 0;
    // defer_rz, the r.z shares are stored and their total is left to the next inverse kernel
    int pq_cnt;
    int defer_rz;
    // V_UPDATE with phic: phi_c += alpha phi_p, the layers of c carried through the
    // iterations (phi_p = W^T p of the iteration's apply, piston left out like the data
    // path), so that the fit needs no inverse transform of the final c
    T* phic;
    const T* phip;
};

enum { V_INIT = 0, V_INIT_WARM = 1, V_UPDATE = 2 };

constexpr int PVEC = 4;     // elements per thread and pass of the vector kernels

// Body of the vector kernel: CTA `cta` of the `nparts` sharing the instance's vectors, NTV
// threads per CTA.
template <class T, int PHASE, int NTV = PBLK>
__device__ __forceinline__ void vec_body(const int n, const VecArgs<T>& v, const int cta,
                                         const int nparts, const int iter_override = -1) {
    const int iter = iter_override >= 0 ? iter_override : v.iter;   // the CG iteration
    __shared__ bool last;
    __shared__ T salpha;
    T ta = T(0);
    bool have_alpha = PHASE != V_UPDATE;
    // The CG update waits for its predecessor (the apply's forward kernel) only after it has
    // issued the loads of c, p, r and J^-1, which that kernel does not write (k_vec launches
    // it without a wait of its own); the other phases were waited for by their caller.
    bool waited = PHASE != V_UPDATE;
    auto form_alpha = [&]() {
        if (threadIdx.x >= 32) return;
        // alpha = rz_k / (p . q)_k; zero if rz vanished (the iterate is final).  Formed
        // once and broadcast (an FP64 division is ~10 instructions on GB300's slow FP64
        // pipe), while the batch's vector loads are in flight; a deferred p.q total first
        // (warp 0, fixed order: the same value in every CTA)
        double pq = 0.0;
        if (v.pq_cnt > 0) {
            pq = warp_total(v.pcg.pqpart + static_cast<long long>(iter) * PQ_SLOTS, v.pq_cnt,
                            static_cast<const DotAcc<T>*>(nullptr));
            if (threadIdx.x == 0 && cta == 0) v.pcg.pqtot[iter] = pq;
        }
        if (threadIdx.x == 0) {
            if (v.pq_cnt == 0) pq = v.pcg.pqtot[iter];
            const double rz = v.pcg.rztot[iter];
            salpha = T((rz != 0.0 && pq > 0.0) ? rz / pq : 0.0);
        }
    };
    DotAcc<T> dot;
    for (int base = cta * NTV * PVEC; base < n; base += nparts * NTV * PVEC) {
        // issue every load of the batch before the arithmetic
        T b[PVEC], q[PVEC], r[PVEC], p[PVEC], c[PVEC], bp[PVEC], jv[PVEC], fc[PVEC], fp[PVEC];
        const bool track = PHASE == V_UPDATE && v.phic != nullptr;
#pragma unroll
        for (int k = 0; k < PVEC; ++k) {
            const int i = base + k * NTV + threadIdx.x;
            if (i < n) {
                jv[k] = v.Jinv[i];
                if (PHASE == V_INIT) {
                    b[k] = v.b[i];
                    q[k] = v.q[i];
                } else if (PHASE == V_INIT_WARM) {
                    b[k] = v.b[i];
                    bp[k] = v.b_prev[i];
                    r[k] = v.r[i];
                } else {
                    c[k] = v.c[i];
                    p[k] = v.p[i];
                    r[k] = v.r[i];
                    if (track) {
                        fc[k] = v.phic[i];
                        fp[k] = v.phip[i];
                    }
                }
            }
        }
        if (!waited) {                   // uniform over the CTA
            pdl_wait();
            pdl_trigger();
            waited = true;
            form_alpha();
        }
        if (PHASE == V_UPDATE) {
#pragma unroll
            for (int k = 0; k < PVEC; ++k) {
                const int i = base + k * NTV + threadIdx.x;
                if (i < n) q[k] = v.q[i];
            }
        }
        if (!have_alpha) {               // uniform over the CTA (base does not depend on the thread)
            __syncthreads();
            ta = salpha;
            have_alpha = true;
        }
#pragma unroll
        for (int k = 0; k < PVEC; ++k) {
            const int i = base + k * NTV + threadIdx.x;
            if (i < n) {
                T rr;
                if (PHASE == V_INIT) {
                    rr = b[k] - q[k];
                    v.b_prev[i] = b[k];
                } else if (PHASE == V_INIT_WARM) {
                    rr = (b[k] - bp[k]) + r[k];
                    v.b_prev[i] = b[k];
                } else {
                    v.c[i] = c[k] + ta * p[k];
                    if (track) v.phic[i] = fc[k] + ta * fp[k];
                    rr = r[k] - ta * q[k];
                }
                v.r[i] = rr;
                const T z = jv[k] * rr;
                v.z[i] = z;
                if (PHASE != V_UPDATE) v.p[i] = z;
                dot.add(rr, z);
            }
        }
    }
    if (!waited) {                       // a CTA without a batch
        pdl_wait();
        pdl_trigger();
    }
    // CTA share of r.z (fixed order), then the last CTA forms the total in a fixed order
    __shared__ double part[NTV];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = (PHASE == V_UPDATE) ? iter + 1 : 0;
    cta_dot_store(dot, part, v.pcg.rzpart + slot * v.pcg.npart + cta);
    if (PHASE == V_UPDATE && v.defer_rz) return;        // the next inverse kernel totals r.z
    if (last_arrival(v.pcg.count, nparts, &last) && w == 0) {
        const double tot = warp_total(v.pcg.rzpart + slot * v.pcg.npart, v.pcg.npart, &dot);
        if (lane == 0) {
            v.pcg.rztot[slot] = tot;
            v.pcg.count[0] = 0;
        }
    }
}

template <class T, int PHASE>
__global__ void __launch_bounds__(PBLK) k_vec(const int n, __grid_constant__ const VecArgs<T> v) {
    if (PHASE != V_UPDATE) pdl_enter();          // V_UPDATE waits inside, after its first loads
    vec_body<T, PHASE>(n, v, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Augmented PCG (Sec. 3.4, the augPCG step of Algorithm 1).  The previous frame's search
// directions P = [p_j] and their images Q = M P (with p_j.q_j) augment this frame's
// Krylov space: the start is corrected over span(P),
//     y_j = p_j.r0 / p_j.q_j,   c0 += sum_j y_j p_j,   r0 -= sum_j y_j q_j,
// and every new direction is made M-conjugate to P,
//     p = z + beta p_old - sum_j mu_j p_j,   mu_j = q_j.z / p_j.q_j.
// Directions of one CG run are M-conjugate, so P^T Q is diagonal.  A direction with
// p_j.q_j <= 0 is skipped.  Vectors in T, inner products and coefficients in double.
// ---------------------------------------------------------------------------
constexpr int AUG_MAX = 8;      // directions kept: the iterations of an augmented frame

enum {
    V_AUG_R0 = 3,        // r0 = b - q (q = M c0), b_prev = b, and p_j.r0
    V_AUG_R0_WARM = 4,   // r0 = (b - b_prev) + r_prev, b_prev = b, and p_j.r0
    V_AUG_INIT = 5,      // c0 += P y, r0 -= Q y, z0 = J^-1 r0, r.z, and q_j.z0
    V_AUG_R0_RESID = 8,  // p_j.r0 of an r0 already formed (the slopes' residual chain)
    V_UPDATE_AUG = 7     // the CG update of V_UPDATE; keeps p.q; q_j.z for the next direction
                         // (the direction update p = z + beta p_old - P mu runs fused into the
                         // inverse wavelet kernel, k_cl_inv with PUPD = 2)
};

template <class T>
struct AugArgs {
    const T* P;          // previous frame's directions, [j * ld + i], j < m
    const T* Q;          // their images M p_j
    const double* pq;    // p_j . q_j
    double* pqnew;       // V_UPDATE_AUG: p.q of this frame's direction `iter`
    double* part;        // [t * npart + cta]: CTA shares of the dots
    double* tot;         // [j]: p_j.r0;  [AUG_MAX + j]: q_j.z
    long long ld;
    int m;               // directions in P, 0 .. AUG_MAX
    int mu_next;         // V_UPDATE_AUG: form q_j.z for the next direction
};

// Warp share of a dot into *dst (lane 0), and the fixed-order total of `nw` warp shares.
__device__ __forceinline__ void warp_share(const DotAcc<double>& a, double* dst) {
    const double x = warp_sum(a.v);
    if ((threadIdx.x & 31) == 0) *dst = x;
}
__device__ __forceinline__ void warp_share(const DotAcc<float>& a, double* dst) {
    const DFloat x = warp_df_sum(DFloat{a.s, a.c});
    if ((threadIdx.x & 31) == 0) *reinterpret_cast<float2*>(dst) = make_float2(x.s, x.c);
}
__device__ __forceinline__ void shares_store(const double* src, int nw, double* slot, const DotAcc<double>*) {
    const int lane = threadIdx.x & 31;
    const double x = warp_sum(lane < nw ? src[lane] : 0.0);
    if (lane == 0) {
        *slot = x;
        __threadfence();
    }
}
__device__ __forceinline__ void shares_store(const double* src, int nw, double* slot, const DotAcc<float>*) {
    const int lane = threadIdx.x & 31;
    const float2 v = lane < nw ? *reinterpret_cast<const float2*>(src + lane) : make_float2(0.f, 0.f);
    const DFloat t = warp_df_sum(DFloat{v.x, v.y});
    if (lane == 0) {
        *reinterpret_cast<float2*>(slot) = make_float2(t.s, t.c);
        __threadfence();
    }
}

template <class T, int PHASE>
__device__ __forceinline__ void aug_body(const int n, const VecArgs<T>& v, const AugArgs<T>& a,
                                         const int cta, const int nparts) {
    constexpr bool R0 = PHASE == V_AUG_R0 || PHASE == V_AUG_R0_WARM || PHASE == V_AUG_R0_RESID;
    __shared__ bool last;
    __shared__ T scoef[AUG_MAX + 1];                 // y_j or mu_j; [AUG_MAX]: alpha or beta
    __shared__ double shares[AUG_MAX + 1][32];       // per-warp shares: [0] r.z, [1 + j] dot j
    const int m = a.m;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = PBLK >> 5;
    // the scalars, one FP64 division per thread (GB300's FP64 pipe is slow)
    if (PHASE == V_AUG_INIT && threadIdx.x < m) {
        const double num = a.tot[threadIdx.x];
        const double den = a.pq[threadIdx.x];
        scoef[threadIdx.x] = T(den > 0.0 ? num / den : 0.0);
    }
    if (PHASE == V_UPDATE_AUG && w == 1) {
        // alpha; a deferred p.q total first (v.pq_cnt > 0: warp 1, fixed order)
        double pq = 0.0;
        if (v.pq_cnt > 0) {
            pq = warp_total(v.pcg.pqpart + static_cast<long long>(v.iter) * PQ_SLOTS, v.pq_cnt,
                            static_cast<const DotAcc<T>*>(nullptr));
        }
        if (lane == 0) {
            if (v.pq_cnt == 0) pq = v.pcg.pqtot[v.iter];
            const double rz = v.pcg.rztot[v.iter];
            scoef[AUG_MAX] = T((rz != 0.0 && pq > 0.0) ? rz / pq : 0.0);
            if (cta == 0) {
                a.pqnew[v.iter] = pq;
                if (v.pq_cnt > 0) v.pcg.pqtot[v.iter] = pq;
            }
        }
    }
    __syncthreads();
    const bool dots = R0 || PHASE == V_AUG_INIT || (PHASE == V_UPDATE_AUG && a.mu_next && m > 0);
    // elements per thread and pass: fewer where a pass holds both P and Q
    constexpr int PV = (PHASE == V_AUG_INIT || sizeof(T) == 8) ? 2 : PVEC;
    DotAcc<T> dj[AUG_MAX];
    DotAcc<T> dot;
    for (int base = cta * PBLK * PV; base < n; base += nparts * PBLK * PV) {
        // every load of the batch before the arithmetic
        T x0[PV], x1[PV], x2[PV], x3[PV], x4[PV];
        T pj[AUG_MAX][PV], qj[AUG_MAX][PV];
#pragma unroll
        for (int k = 0; k < PV; ++k) {
            const int i = base + k * PBLK + threadIdx.x;
            if (i < n) {
                if (PHASE == V_AUG_R0) {
                    x0[k] = v.b[i];
                    x1[k] = v.q[i];
                } else if (PHASE == V_AUG_R0_WARM) {
                    x0[k] = v.b[i];
                    x1[k] = v.b_prev[i];
                    x2[k] = v.r[i];
                } else if (PHASE == V_AUG_R0_RESID) {
                    x0[k] = v.r[i];
                } else if (PHASE == V_AUG_INIT) {
                    x0[k] = v.c[i];
                    x1[k] = v.r[i];
                    x2[k] = v.Jinv[i];
                } else {
                    x0[k] = v.c[i];
                    x1[k] = v.p[i];
                    x2[k] = v.r[i];
                    x3[k] = v.q[i];
                    x4[k] = v.Jinv[i];
                }
#pragma unroll
                for (int j = 0; j < AUG_MAX; ++j) {
                    if (j < m) {
                        if (R0 || PHASE == V_AUG_INIT) pj[j][k] = a.P[j * a.ld + i];
                        if (PHASE == V_AUG_INIT || (PHASE == V_UPDATE_AUG && dots)) qj[j][k] = a.Q[j * a.ld + i];
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PV; ++k) {
            const int i = base + k * PBLK + threadIdx.x;
            if (i < n) {
                if (R0) {
                    const T rr = PHASE == V_AUG_R0 ? x0[k] - x1[k]
                                 : PHASE == V_AUG_R0_WARM ? (x0[k] - x1[k]) + x2[k] : x0[k];
                    if (PHASE != V_AUG_R0_RESID) {
                        v.r[i] = rr;
                        v.b_prev[i] = x0[k];
                    }
#pragma unroll
                    for (int j = 0; j < AUG_MAX; ++j)
                        if (j < m) dj[j].add(pj[j][k], rr);
                } else if (PHASE == V_AUG_INIT) {
                    T c = x0[k], rr = x1[k];
#pragma unroll
                    for (int j = 0; j < AUG_MAX; ++j) {
                        if (j < m) {
                            c += scoef[j] * pj[j][k];
                            rr -= scoef[j] * qj[j][k];
                        }
                    }
                    const T z = x2[k] * rr;
                    v.c[i] = c;
                    v.r[i] = rr;
                    v.z[i] = z;
                    dot.add(rr, z);
#pragma unroll
                    for (int j = 0; j < AUG_MAX; ++j)
                        if (j < m) dj[j].add(qj[j][k], z);

                } else {
                    const T al = scoef[AUG_MAX];
                    v.c[i] = x0[k] + al * x1[k];
                    const T rr = x2[k] - al * x3[k];
                    const T z = x4[k] * rr;
                    v.r[i] = rr;
                    v.z[i] = z;
                    dot.add(rr, z);
                    if (dots) {
#pragma unroll
                        for (int j = 0; j < AUG_MAX; ++j)
                            if (j < m) dj[j].add(qj[j][k], z);
                    }
                }
            }
        }
    }
    // CTA shares (fixed order): t = 0 is r.z (not in the R0 phases), t = 1 + j dot j
    const bool has_rz = !R0;
    const int nd = dots ? m : 0;
    if (has_rz) warp_share(dot, &shares[0][w]);
#pragma unroll
    for (int j = 0; j < AUG_MAX; ++j)
        if (j < nd) warp_share(dj[j], &shares[1 + j][w]);
    __syncthreads();
    const int slot = PHASE == V_UPDATE_AUG ? v.iter + 1 : 0;
    for (int t = w; t <= nd; t += nw) {
        if (t == 0 && !has_rz) continue;
        double* dst = t == 0 ? v.pcg.rzpart + slot * v.pcg.npart + cta : a.part + (t - 1) * v.pcg.npart + cta;
        shares_store(shares[t], nw, dst, &dot);
    }
    // deferred: the next inverse kernel totals r.z and the q_j.z dots
    if (PHASE == V_UPDATE_AUG && v.defer_rz) return;
    if (last_arrival(v.pcg.count, nparts, &last)) {
        // the totals, one warp each, in a fixed order over the CTAs
        for (int t = w; t <= nd; t += nw) {
            if (t == 0 && !has_rz) continue;
            const double* src = t == 0 ? v.pcg.rzpart + slot * v.pcg.npart : a.part + (t - 1) * v.pcg.npart;
            const double tot = warp_total(src, v.pcg.npart, &dot);
            if (lane == 0) {
                if (t == 0)
                    v.pcg.rztot[slot] = tot;
                else
                    a.tot[(R0 ? 0 : AUG_MAX) + t - 1] = tot;
            }
        }
        if (threadIdx.x == 0) v.pcg.count[0] = 0;
    }
}

template <class T, int PHASE>
__global__ void __launch_bounds__(PBLK) k_aug(const int n, __grid_constant__ const VecArgs<T> v,
                                              __grid_constant__ const AugArgs<T> a) {
    pdl_enter();
    aug_body<T, PHASE>(n, v, a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// DM fitting (Algorithm 1 fitting step, Table 3): a~_m(p, q) = sum_l w_lm phi_l
// sampled bilinearly at the actuator, then the control law of Algorithm 1: open loop
// (apply_gain 1) a = (1-g) a_prev + g a~; closed loop (apply_gain 2)
// a = a_prev + g (a~ - a_old), after which a_old = a_prev (the commands of the frame
// before) and a_prev = a.
// ---------------------------------------------------------------------------
template <class T, int NTF = PBLK>
__device__ __forceinline__ void fit_body(const Desc<T>& d, const T* __restrict__ phi,
                                         T* __restrict__ a_prev, T* __restrict__ out, int apply_gain,
                                         const int blk, T* __restrict__ a_old = nullptr,
                                         const T* __restrict__ cpist = nullptr) {
    const int idx = blk * NTF + threadIdx.x;
    if (idx >= d.n_act) return;
    int m = 0;
    while (m + 1 < d.n_dms && idx >= d.Mi[m + 1].off) ++m;
    const int na = d.Mi[m].n_act, loc = idx - d.Mi[m].off;
    const int p = loc / na, q = loc - p * na;
    // layers four at a time: their table loads, then their samples, all in flight
    // together; the terms are added in layer order
    T acc = T(0);
    for (int l0 = 0; l0 < d.n_layers; l0 += 4) {
        T w[4], fy[4], fx[4], v[4][4];
        int i0[4], j0[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int l = l0 + u;
            w[u] = l < d.n_layers ? d.fitw[m][l] : T(0);
            if (w[u] != T(0)) {
                const int tb = (m * MAXL + l) * MAXNACT;
                i0[u] = d.di0[tb + p];
                j0[u] = d.di0[tb + q];
                fy[u] = d.dfw[tb + p];
                fx[u] = d.dfw[tb + q];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (w[u] != T(0)) {
                const int l = l0 + u, n = d.L[l].n;
                const T* P = phi + d.L[l].off + i0[u] * n + j0[u];
                v[u][0] = P[0];
                v[u][1] = P[1];
                v[u][2] = P[n];
                v[u][3] = P[n + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (w[u] != T(0))
                acc += w[u] * ((T(1) - fy[u]) * ((T(1) - fx[u]) * v[u][0] + fx[u] * v[u][1]) +
                               fy[u] * ((T(1) - fx[u]) * v[u][2] + fx[u] * v[u][3]));
    }
    if (cpist) {
        // phi without the full layers' pistons (the carried layers): a unit piston coefficient
        // synthesises to 1/n on every node of an n x n layer, and the bilinear weights sum
        // to one, so each adds w_lm c_piston / n
        for (int l = 0; l < d.n_layers; ++l) {
            const T wl = d.fitw[m][l];
            if (d.L[l].full && wl != T(0)) acc += wl * (cpist[d.L[l].off] / T(d.L[l].n));
        }
    }
    if (apply_gain == 2) {
        const T cur = a_prev[idx];
        const T a = cur + d.gain * (acc - a_old[idx]);
        a_old[idx] = cur;
        a_prev[idx] = a;
        out[idx] = a;
    } else if (apply_gain) {
        const T a = (T(1) - d.gain) * a_prev[idx] + d.gain * acc;
        a_prev[idx] = a;
        out[idx] = a;
    } else {
        out[idx] = acc;
    }
}

template <class T>
__global__ void __launch_bounds__(PBLK) k_fit(__grid_constant__ const Desc<T> d, const T* __restrict__ phi,
                                              T* __restrict__ a_prev, T* __restrict__ out,
                                              int apply_gain, T* __restrict__ a_old,
                                              const T* __restrict__ cpist) {
    pdl_enter();
    fit_body<T>(d, phi, a_prev, out, apply_gain, blockIdx.x, a_old, cpist);
}

// ---------------------------------------------------------------------------
// Pseudo-open-loop slopes of the closed loop (Algorithm 1): s_pol = s + Gamma P_DM a with
// a the commands of two frames back (the two-step delay).  The DM shape is bilinear
// between actuators (Sec. 4.1), i.e. zero beyond the outer actuators' hats; sensor g sees
// DM m at s x + theta h_m, like a layer.  Two kernels: the DM shapes on every aperture
// node, then the slopes; block (x, g) of the second takes PBLK of sensor g's fine
// subapertures, or, on a coarse sensor, coarse subaperture x ((1/nb) x the sum of its
// active fine slopes, R9).
// ---------------------------------------------------------------------------
template <class T>
struct PolArgs {
    const T* s;          // measured (residual) slopes
    const T* a;          // the commands a^(i-1)
    T* out;              // pseudo-open-loop slopes
    T* nodes;            // the DM shapes on the aperture nodes (n_nodes)
    const int* qi0y;     // DM tables, pair (g, m) at (g * MAXM + m) * TAB
    const int* qi0x;
    const T* qfy;
    const T* qfx;
};

// The DM shapes seen by sensor g at aperture node (row ra, column cb).
template <class T>
__device__ __forceinline__ T dm_node(const Desc<T>& d, const PolArgs<T>& p, int g, int ra, int cb) {
    T v = T(0);
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
        if (m >= d.n_dms) break;
        const int base = (g * MAXM + m) * TAB;
        const int iy = p.qi0y[base + ra], ix = p.qi0x[base + cb];
        const T fy = p.qfy[base + ra], fx = p.qfx[base + cb];
        const int na = d.Mi[m].n_act;
        const T* A = p.a + d.Mi[m].off;
        const bool y0 = iy >= 0 && iy < na, y1 = iy + 1 >= 0 && iy + 1 < na;
        const bool x0 = ix >= 0 && ix < na, x1 = ix + 1 >= 0 && ix + 1 < na;
        const T a00 = (y0 && x0) ? A[iy * na + ix] : T(0);
        const T a01 = (y0 && x1) ? A[iy * na + ix + 1] : T(0);
        const T a10 = (y1 && x0) ? A[(iy + 1) * na + ix] : T(0);
        const T a11 = (y1 && x1) ? A[(iy + 1) * na + ix + 1] : T(0);
        v += (T(1) - fy) * ((T(1) - fx) * a00 + fx * a01) + fy * ((T(1) - fx) * a10 + fx * a11);
    }
    return v;
}

// The DM shapes on every aperture node of every sensor, one thread per node.
template <class T>
__global__ void __launch_bounds__(PBLK) k_dmnodes(__grid_constant__ const Desc<T> d,
                                                  __grid_constant__ const PolArgs<T> p) {
    pdl_enter();
    const int k = blockIdx.x * PBLK + threadIdx.x;
    if (k >= d.n_nodes) return;
    int g = 0;
    while (g + 1 < d.n_wfs && k >= d.G[g + 1].node_off) ++g;
    const int np = d.G[g].N + 1, loc = k - d.G[g].node_off;
    const int ra = loc / np, cb = loc - ra * np;
    p.nodes[k] = dm_node(d, p, g, ra, cb);
}

// Gamma of node values v (row stride np) on fine subaperture (i, j) (Sec. 2, reading R1
// for s^y).
template <class T>
__device__ __forceinline__ void node_slope(const T* v, int np, int i, int j, T& sx, T& sy) {
    const T v00 = v[i * np + j], v01 = v[i * np + j + 1];
    const T v10 = v[(i + 1) * np + j], v11 = v[(i + 1) * np + j + 1];
    sx = T(0.5) * ((v01 - v00) + (v11 - v10));
    sy = T(0.5) * ((v10 - v00) + (v11 - v01));
}

constexpr int POLBLK = 1024;   // threads of the slope kernel: a coarse block in 2 passes

template <class T>
__global__ void __launch_bounds__(POLBLK) k_pol(__grid_constant__ const Desc<T> d,
                                                __grid_constant__ const PolArgs<T> p) {
    pdl_enter();
    const int g = blockIdx.y;
    const WfsInfo& W = d.G[g];
    const int N = W.N, np = N + 1;
    const T* v = p.nodes + W.node_off;
    if (W.nb == 1) {
        const int k = blockIdx.x * POLBLK + threadIdx.x;
        if (k >= N * N) return;
        const int id = d.sidx[W.mask_off + k];
        if (id < 0) return;
        const int i = k / N, j = k - i * N;
        T sx, sy;
        node_slope(v, np, i, j, sx, sy);
        p.out[W.soff + id] = p.s[W.soff + id] + sx;
        p.out[W.soff + W.n_active + id] = p.s[W.soff + W.n_active + id] + sy;
        return;
    }
    const int K = blockIdx.x;
    if (K >= W.n_sub * W.n_sub) return;
    const int cid = d.cidx[W.cmask_off + K];
    if (cid < 0) return;                                  // uniform over the block
    const int I = K / W.n_sub, J = K - I * W.n_sub, nb = W.nb;
    T ax = T(0), ay = T(0);
    for (int t = threadIdx.x; t < nb * nb; t += POLBLK) {
        const int u = t / nb, w = t - u * nb;
        const int i = I * nb + u, j = J * nb + w;
        // the node loads do not wait for the mask (every (i, j) of the block is inside)
        T sx, sy;
        node_slope(v, np, i, j, sx, sy);
        if (d.sidx[W.mask_off + i * N + j] == cid) {
            ax += sx;
            ay += sy;
        }
    }
    // fixed-order block sum
    __shared__ T sh[2][POLBLK / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        ax += __shfl_down_sync(0xffffffffu, ax, o);
        ay += __shfl_down_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) {
        sh[0][w] = ax;
        sh[1][w] = ay;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T tx = T(0), ty = T(0);
        for (int k = 0; k < POLBLK / 32; ++k) {
            tx += sh[0][k];
            ty += sh[1][k];
        }
        p.out[W.soff + cid] = p.s[W.soff + cid] + tx / T(nb);
        p.out[W.soff + W.n_active + cid] = p.s[W.soff + W.n_active + cid] + ty / T(nb);
    }
}

// ---------------------------------------------------------------------------
// Per-layer sums S_l = sum over layer l of lambda_i D_i c_i, in double, one CTA per
// layer in a fixed order: the gradients of the converged reconstruction with respect to
// alpha (-sum_l S_l) and to the layer Cn2 weights (alpha S_l / w_l), since
// dM/dalpha = D and D_l is proportional to 1 / w_l (Sec. 3.1 prior).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(PBLK) k_layer_dots(__grid_constant__ const Desc<T> d, const T* __restrict__ lam,
                                                     const T* __restrict__ c, double* __restrict__ out) {
    __shared__ double part[PBLK];
    const int l = blockIdx.x;
    const int off = d.L[l].off, n2 = d.L[l].n * d.L[l].n;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n2; i += PBLK)
        acc += double(lam[off + i]) * double(d.D[off + i]) * double(c[off + i]);
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = 0.0;
        for (int k = threadIdx.x; k < PBLK; k += 32) x += part[k];
        x = warp_sum(x);
        if (threadIdx.x == 0) out[l] = x;
    }
}

// out = a x + b y + c (u o v) elementwise, a null pointer dropping its term (out may be x
// or y): the double residual b - M x of the mixed-precision converged solves.
template <class T>
__global__ void __launch_bounds__(PBLK) k_lin(const int n, const double a, const T* x, const double b, const T* y,
                                              const double c, const T* u, const T* v, T* out) {
    const T ta = T(a), tb = T(b), tc = T(c);
    for (int i = blockIdx.x * PBLK + threadIdx.x; i < n; i += gridDim.x * PBLK) {
        T acc = T(0);
        if (x) acc = ta * x[i];
        if (y) acc += tb * y[i];
        if (u) acc += tc * (u[i] * v[i]);
        out[i] = acc;
    }
}


// ---------------------------------------------------------------------------
// Reverse pass through the fixed-iteration frame with its scalars on the device (a build
// addition).  Iteration i of the PCG recurrence (Sec. 3.3) is run backwards, statement by
// statement, in three vector kernels around one M-apply (M and J^-1 are symmetric):
//   VJ_A  p_bar = pi_bar + M q_bar (of iteration i + 1; not for the first), z_bar = p_bar,
//         pi_bar = beta_i p_bar, beta_bar = p_bar . p_i, then rho_bar += beta_bar / rho_i and
//         rho_bar_i = -beta_bar rho_(i+1) / rho_i^2;
//   VJ_B  r_bar += rho_bar z_(i+1), z_bar += rho_bar r_(i+1), r_bar += J^-1 z_bar, then
//         alpha_bar = -r_bar . q_i + c_bar . p_i, rho_bar_i += alpha_bar / sigma_i and
//         sigma_bar = -alpha_bar rho_i / sigma_i^2;
//   VJ_C  q_bar = -alpha_i r_bar + sigma_bar p_i, pi_bar += alpha_i c_bar + sigma_bar q_i
//         (q_bar then goes through M);
//   VJ_E  after iteration 0: p_bar = pi_bar + M q_bar, rho_bar = rho_bar_0, z_bar = p_bar,
//         r_bar += rho_bar z_0, z_bar += rho_bar r_0, r_bar += J^-1 z_bar (r_bar = b_bar).
// rho_i = r_i.z_i and sigma_i = p_i.q_i are the forward pass's own totals (rz and p.q slots).
// The scalar adjoints live in rs[0] (rho_bar), rs[1] (rho_bar_i), rs[2] (sigma_bar); the
// inner products are fixed-order CTA shares totalled by the last CTA to arrive.
// ---------------------------------------------------------------------------
enum { VJ_A = 0, VJ_B = 1, VJ_C = 2, VJ_E = 3 };

template <class T>
struct VjpArgs {
    T* rbar;
    T* pbar;
    T* pbi;
    T* qbar;
    const T* cbar;
    const T* Mq;         // M q_bar of the previous reverse iteration (VJ_A not first, VJ_E)
    const T* Jinv;
    const T* p;          // p_i
    const T* q;          // q_i
    const T* r1;         // r_(i+1) (VJ_E: r_0)
    const T* z1;         // z_(i+1) (VJ_E: z_0)
    const double* rho;   // rho_0 .. rho_k
    const double* sigma; // sigma_0 .. sigma_(k-1)
    double* rs;          // scalar adjoints
    double* part;        // CTA shares: [0 .. NPART) and [NPART .. 2 NPART)
    unsigned* count;     // arrival counter, reset by the last CTA
    int i;
    int first;           // VJ_A: the first reverse iteration (p_bar = 0, nothing to add)
    int npart;           // stride of the share slots
};

template <class T, int PHASE>
__global__ void __launch_bounds__(PBLK) k_vjp(const int n, __grid_constant__ const VjpArgs<T> v) {
    __shared__ bool last;
    __shared__ double part[PBLK];
    __shared__ T sc[4];
    const int i = v.i;
    if (threadIdx.x == 0) {
        // the CTA's scalar coefficients, formed once in double
        const double rho = v.rho[PHASE == VJ_E ? 0 : i];
        if (PHASE == VJ_A) sc[0] = T(v.rho[i + 1] / rho);                     // beta_i
        if (PHASE == VJ_B) sc[0] = T(v.rs[0]);                                // rho_bar
        if (PHASE == VJ_C) {
            sc[0] = T(rho / v.sigma[i]);                                      // alpha_i
            sc[1] = T(v.rs[2]);                                               // sigma_bar
        }
        if (PHASE == VJ_E) sc[0] = T(v.rs[1]);                                // rho_bar_0
    }
    __syncthreads();
    DotAcc<T> d1, d2;
    for (int k = blockIdx.x * PBLK + threadIdx.x; k < n; k += gridDim.x * PBLK) {
        if (PHASE == VJ_A) {
            const T pb = v.first ? T(0) : v.pbi[k] + v.Mq[k];
            if (!v.first) v.pbar[k] = pb;
            v.pbi[k] = sc[0] * pb;
            d1.add(pb, v.p[k]);
        } else if (PHASE == VJ_B) {
            const T rb = v.rbar[k] + sc[0] * v.z1[k];
            const T zb = v.pbar[k] + sc[0] * v.r1[k];
            const T r2 = rb + v.Jinv[k] * zb;
            v.rbar[k] = r2;
            d1.add(r2, v.q[k]);
            d2.add(v.cbar[k], v.p[k]);
        } else if (PHASE == VJ_C) {
            const T qb = -sc[0] * v.rbar[k];
            v.qbar[k] = qb + sc[1] * v.p[k];
            const T pb = v.pbi[k] + sc[0] * v.cbar[k];
            v.pbi[k] = pb + sc[1] * v.q[k];
        } else {
            const T pb = v.pbi[k] + v.Mq[k];
            const T rb = v.rbar[k] + sc[0] * v.z1[k];
            const T zb = pb + sc[0] * v.r1[k];
            v.rbar[k] = rb + v.Jinv[k] * zb;
        }
    }
    if (PHASE != VJ_A && PHASE != VJ_B) return;
    cta_dot_store(d1, part, v.part + blockIdx.x);
    if (PHASE == VJ_B) cta_dot_store(d2, part, v.part + v.npart + blockIdx.x);
    if (last_arrival(v.count, gridDim.x, &last) && threadIdx.x < 32) {
        const double t1 = warp_total(v.part, gridDim.x, &d1);
        const double t2 = PHASE == VJ_B ? warp_total(v.part + v.npart, gridDim.x, &d2) : 0.0;
        if (threadIdx.x == 0) {
            const double rho = v.rho[i], rho1 = v.rho[i + 1];
            if (PHASE == VJ_A) {
                const double rb = v.first ? v.rs[0] : v.rs[1];                // rho_bar carried in
                v.rs[0] = rb + t1 / rho;
                v.rs[1] = -t1 * rho1 / (rho * rho);
            } else {
                const double sig = v.sigma[i], abar = -t1 + t2;
                v.rs[1] += abar / sig;
                v.rs[2] = -abar * rho / (sig * sig);
            }
            v.count[0] = 0;
        }
    }
}

// b^T J^-1 b in double, one CTA, fixed order (the reference of a warm-started solve's
// relative residual).
template <class T>
__global__ void __launch_bounds__(PBLK) k_wnorm(const int n, const T* __restrict__ b, const T* __restrict__ jinv,
                                                double* __restrict__ out) {
    __shared__ double part[PBLK];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += PBLK) acc += double(b[i]) * double(b[i]) * double(jinv[i]);
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = 0.0;
        for (int k = threadIdx.x; k < PBLK; k += 32) x += part[k];
        x = warp_sum(x);
        if (threadIdx.x == 0) *out = x;
    }
}

// ---------------------------------------------------------------------------
// Reliable updates of a mixed-precision CG (a build addition for the converged solves of
// the single-precision form): the recurrence runs in T on a residual scaled to unit
// J^-1-norm, its iterate is an increment x that is folded into the double iterate x64
// (x64 += sc x, x = 0) whenever the recurrence's residual has dropped tenfold; the true
// residual b - M x64 is then formed in double and replaces the recurrence's residual
// (r = T(r64 / sc_new), z = J^-1 r, p scaled by sc_old / sc_new so that the search
// direction continues).  r.z of the refreshed residual goes to rz slot `slot` (0 on a
// restart, where also p = z; 1 otherwise, with slot 0 set to rz0, the previous r.z in
// the new scale, so that the next direction update forms beta = slot 1 / slot 0).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(PBLK) k_accum(const int n, const double sc, T* __restrict__ x,
                                                double* __restrict__ x64) {
    for (int i = blockIdx.x * PBLK + threadIdx.x; i < n; i += gridDim.x * PBLK) {
        x64[i] += sc * double(x[i]);
        x[i] = T(0);
    }
}

template <class T>
__global__ void __launch_bounds__(PBLK) k_refresh(const int n, const double* __restrict__ r64, const double scale,
                                                  const double ratio, const int restart, const double rz0,
                                                  __grid_constant__ const VecArgs<T> v) {
    __shared__ bool last;
    __shared__ double part[PBLK];
    const int cta = blockIdx.x, nparts = gridDim.x;
    const T tr = T(ratio);
    DotAcc<T> dot;
    for (int i = cta * PBLK + threadIdx.x; i < n; i += nparts * PBLK) {
        const T r = T(scale * r64[i]);
        const T z = v.Jinv[i] * r;
        v.r[i] = r;
        v.z[i] = z;
        v.p[i] = restart ? z : tr * v.p[i];
        dot.add(r, z);
    }
    const int slot = restart ? 0 : 1;
    cta_dot_store(dot, part, v.pcg.rzpart + slot * v.pcg.npart + cta);
    if (last_arrival(v.pcg.count, nparts, &last) && threadIdx.x < 32) {
        const double tot = warp_total(v.pcg.rzpart + slot * v.pcg.npart, v.pcg.npart, &dot);
        if (threadIdx.x == 0) {
            v.pcg.rztot[slot] = tot;
            if (!restart) v.pcg.rztot[0] = rz0;
            v.pcg.count[0] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Exact Jacobi diagonal of W B W^T (Eq. 7), one warp per wavelet coefficient, in
// double.  The basis function of coefficient (layer l, row r, col c) is the outer
// product f_y(i) f_x(j) of 1-D level-j functions (shifted copies of the tables), its
// bilinear projection on sensor g is (Ry f_y)(Rx f_x)^T, and its slopes are
// products of 1-D averages and differences:
//   s^x(i, j) = avg_y(i) dif_x(j),  s^y(i, j) = dif_y(i) avg_x(j).
// The diagonal is sigma^-2 * (sum of squared active slopes, minus the squared
// tip/tilt means times |M| for an LGS; or the sum of squared coarse slopes).
// ---------------------------------------------------------------------------
struct DiagArgs {
    const double* basis;
    const int* basis_off;
    const double* pfy;   // projection weights in double (same layout as Desc::pfy)
    const double* pfx;
    double* out;         // n_c
};

template <class T>
__global__ void __launch_bounds__(128) k_jdiag(const Desc<T> d, const DiagArgs a) {
    __shared__ double sF[4][TAB];
    __shared__ double sG[4][TAB];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int coef = blockIdx.x * 4 + w;
    if (coef >= d.n_c) return;
    int l = 0;
    while (l + 1 < d.n_layers && coef >= d.L[l + 1].off) ++l;
    const LayerInfo L = d.L[l];
    const int n = L.n, k = coef - L.off, r = k >> L.log2n, c = k & (n - 1);
    const int mx = r > c ? r : c;
    int j, ky, kx, sy, sx;
    if (mx < (n >> L.levels)) {
        j = L.levels;
        ky = kx = 0;
        sy = r;
        sx = c;
    } else {
        j = L.log2n - (31 - __clz(mx));
        const int h = n >> j;
        ky = r >= h;
        kx = c >= h;
        sy = r - ky * h;
        sx = c - kx * h;
    }
    const double* fy = a.basis + a.basis_off[basis_index(l, j, ky)];
    const double* fx = a.basis + a.basis_off[basis_index(l, j, kx)];
    const int shy = sy << j, shx = sx << j;
    double* F = sF[w];
    double* G = sG[w];
    double total = 0.0;
    for (int g = 0; g < d.n_wfs; ++g) {
        const WfsInfo W = d.G[g];
        const int N = W.N, NP = N + 1;
        const int tp = (g * MAXL + l) * TAB;
        int lo_a = NP, hi_a = -1, lo_b = NP, hi_b = -1;
        for (int t = lane; t < NP; t += 32) {
            const int i0 = d.pi0y[tp + t];
            const double wy = a.pfy[tp + t];
            const double v = (1.0 - wy) * fy[(i0 - shy) & (n - 1)] + wy * fy[(i0 + 1 - shy) & (n - 1)];
            F[t] = v;
            if (v != 0.0) {
                lo_a = min(lo_a, t);
                hi_a = max(hi_a, t);
            }
            const int j0 = d.pi0x[tp + t];
            const double wx = a.pfx[tp + t];
            const double u = (1.0 - wx) * fx[(j0 - shx) & (n - 1)] + wx * fx[(j0 + 1 - shx) & (n - 1)];
            G[t] = u;
            if (u != 0.0) {
                lo_b = min(lo_b, t);
                hi_b = max(hi_b, t);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            lo_a = min(lo_a, __shfl_xor_sync(0xffffffffu, lo_a, o));
            hi_a = max(hi_a, __shfl_xor_sync(0xffffffffu, hi_a, o));
            lo_b = min(lo_b, __shfl_xor_sync(0xffffffffu, lo_b, o));
            hi_b = max(hi_b, __shfl_xor_sync(0xffffffffu, hi_b, o));
        }
        __syncwarp();
        if (hi_a < 0 || hi_b < 0) {
            __syncwarp();
            continue;
        }
        // subaperture rows i use nodes i, i+1
        const int i0 = max(lo_a - 1, 0), i1 = min(hi_a, N - 1);
        const int j0 = max(lo_b - 1, 0), j1 = min(hi_b, N - 1);
        const int wi = i1 - i0 + 1, wj = j1 - j0 + 1;
        const int* sidx = d.sidx + W.mask_off;
        double contrib = 0.0;
        if (W.nb == 1) {
            double s2 = 0.0, tx = 0.0, ty = 0.0, E = 0.0, e1 = 0.0, e2 = 0.0;
            if (wi > 0 && wj > 0) {
                for (int t = lane; t < wi * wj; t += 32) {
                    const int i = i0 + t / wj, jj = j0 + t % wj;
                    if (sidx[i * N + jj] < 0) continue;
                    const double ya = 0.5 * (F[i] + F[i + 1]), yd = F[i + 1] - F[i];
                    const double xa = 0.5 * (G[jj] + G[jj + 1]), xd = G[jj + 1] - G[jj];
                    const double vx = ya * xd, vy = yd * xa;
                    s2 += vx * vx + vy * vy;
                    tx += vx;
                    ty += vy;
                    if (W.el) {
                        double b1, b2, gam;
                        elong(W, i, jj, b1, b2, gam);
                        const double bv = b1 * vx + b2 * vy;
                        E += gam * bv * bv;
                        e1 += gam * b1 * bv;
                        e2 += gam * b2 * bv;
                    }
                }
            }
            s2 = warp_sum(s2);
            tx = warp_sum(tx);
            ty = warp_sum(ty);
            contrib = s2;
            if (W.lgs) contrib -= (tx * tx + ty * ty) / W.n_active;
            if (W.el) {
                // minus the elongation term: sum of gamma (beta . u)^2 over the mask, u the
                // slopes without their means m = (tx, ty) / |M|: E - 2 m . e + m^T K m
                E = warp_sum(E);
                e1 = warp_sum(e1);
                e2 = warp_sum(e2);
                const double mx = tx / W.n_active, my = ty / W.n_active;
                contrib -= E - 2.0 * (mx * e1 + my * e2) +
                           (W.el_K11 * mx * mx + 2.0 * W.el_K12 * mx * my + W.el_K22 * my * my);
            }
        } else {
            const int ns = W.n_sub, nb = W.nb;
            for (int blk = 0; blk < ns * ns; ++blk) {
                if (d.cidx[W.cmask_off + blk] < 0) continue;
                const int I = blk / ns, J = blk - I * ns;
                const int bi0 = max(i0, I * nb), bi1 = min(i1, I * nb + nb - 1);
                const int bj0 = max(j0, J * nb), bj1 = min(j1, J * nb + nb - 1);
                double cx = 0.0, cy = 0.0;
                if (bi0 <= bi1 && bj0 <= bj1) {
                    const int bw = bj1 - bj0 + 1, cnt = (bi1 - bi0 + 1) * bw;
                    for (int t = lane; t < cnt; t += 32) {
                        const int i = bi0 + t / bw, jj = bj0 + t % bw;
                        if (sidx[i * N + jj] < 0) continue;
                        const double ya = 0.5 * (F[i] + F[i + 1]), yd = F[i + 1] - F[i];
                        const double xa = 0.5 * (G[jj] + G[jj + 1]), xd = G[jj + 1] - G[jj];
                        cx += ya * xd;
                        cy += yd * xa;
                    }
                }
                cx = warp_sum(cx) / nb;
                cy = warp_sum(cy) / nb;
                contrib += cx * cx + cy * cy;
            }
        }
        total += W.sig2inv * contrib;
        __syncwarp();
    }
    if (lane == 0) a.out[coef] = total;
}

// J = data diagonal + alpha max(D, tau); Jinv in the handle's type.
template <class T>
__global__ void k_jfinish(int n, const double* __restrict__ data, const double* __restrict__ D,
                          double alpha, double tau, T* __restrict__ Jinv, T* __restrict__ Dt,
                          double* __restrict__ J) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double j = data[i] + alpha * (D[i] > tau ? D[i] : tau);
    J[i] = j;
    Jinv[i] = T(1.0 / j);
    Dt[i] = T(D[i]);
}

template <class T, class U>
__global__ void k_convert(int n, const U* __restrict__ in, T* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = T(in[i]);
}

}  // namespace fewha
