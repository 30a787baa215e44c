// Cluster kernels of the FEWHA hot path: one thread-block cluster of CL CTAs per layer
// (wavelet transforms with the adjoint projection) and per sensor (projection, slopes,
// noise weighting, adjoint slopes).  The CTAs of a cluster split the work into bands
// and exchange data through distributed shared memory; every reduction runs in a fixed
// order, so results stay bitwise reproducible.  Global reads are staged into shared
// memory with cp.async so that all of a CTA's loads are in flight at once.
#pragma once

#include <cooperative_groups.h>

#include "fewha_kernels.cuh"

namespace fewha {

namespace cg = cooperative_groups;

constexpr int CL = 8;        // CTAs per cluster
constexpr int RMAX = 8;      // wavelet pairs per thread and pass
constexpr int CWMAX = 16;    // warps per CTA at most
constexpr int RED_DBL = 520; // reduction scratch at the head of shared memory, in doubles

// Threads per CTA: 512 in single precision (latency hiding), 256 in double precision
// (the register budget of the sliding windows).
template <class T>
__host__ __device__ constexpr int cblk() {
    return sizeof(T) == 4 ? 512 : 256;
}

// ---------------------------------------------------------------- cp.async staging
template <class T>
__device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// 16-byte copy; both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
// Elements per 16-byte chunk.
template <class T>
__host__ __device__ constexpr int vec16() {
    return 16 / static_cast<int>(sizeof(T));
}
// The 16-byte vector of T and its element access.
template <class T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static __device__ __forceinline__ float at(const float4& v, int e) {
        return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
    }
};
template <> struct Vec16<double> {
    using type = double2;
    static __device__ __forceinline__ double at(const double2& v, int e) { return e == 0 ? v.x : v.y; }
};

// Stage `count` elements from src to dst (both 16-byte aligned) in 16-byte chunks by the
// threads [t0, t0 + nthr); reads up to one chunk past src + count (allocations are padded).
template <class T>
__device__ __forceinline__ void stage16(T* dst, const T* src, int count, int t, int nthr) {
    constexpr int V = vec16<T>();
    const int chunks = (count + V - 1) / V;
    for (int c = t; c < chunks; c += nthr) cp_async16(dst + c * V, src + c * V);
}

// ---------------------------------------------------------------- one db3 step
// One periodic db3 analysis (INV = false) or synthesis (INV = true) step along an axis
// of `lines` independent lines of length m, in place.  Element (line, pos) lives at
// buf[line * ls + pos * ps].  A thread owns a run of R consecutive pairs of one line and
// keeps a sliding window of the inputs in registers.  R is a compile-time constant of
// the code that runs (1, 2, 4 or 8): the small coarse levels have R = 1, and code
// unrolled for the largest R under run-time predicates made them instruction-bound.
// WARP: the pass is run by one warp alone, which synchronises with __syncwarp.
template <class T, bool INV, int R, bool WARP = false>
__device__ __forceinline__ void dwt_run(T* Lp, int m, int h, int k0, int ps, bool act) {
    T o0[R], o1[R];
    if (act) {
        if (!INV) {
            T w[2 * R + 4];
#pragma unroll
            for (int s = 0; s < 2 * R + 4; ++s) w[s] = Lp[((2 * k0 + s) & (m - 1)) * ps];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                T a = T(0), d = T(0);
#pragma unroll
                for (int tt = 0; tt < 6; ++tt) {
                    a += tap_h<T>(tt) * w[2 * q + tt];
                    d += tap_g<T>(tt) * w[2 * q + tt];
                }
                o0[q] = a;
                o1[q] = d;
            }
        } else {
            T wa[R + 2], wd[R + 2];
#pragma unroll
            for (int s = 0; s < R + 2; ++s) {
                const int idx = (k0 - 2 + s) & (h - 1);
                wa[s] = Lp[idx * ps];
                wd[s] = Lp[(h + idx) * ps];
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
                o0[q] = tap_h<T>(0) * wa[q + 2] + tap_h<T>(2) * wa[q + 1] + tap_h<T>(4) * wa[q] +
                        tap_g<T>(0) * wd[q + 2] + tap_g<T>(2) * wd[q + 1] + tap_g<T>(4) * wd[q];
                o1[q] = tap_h<T>(1) * wa[q + 2] + tap_h<T>(3) * wa[q + 1] + tap_h<T>(5) * wa[q] +
                        tap_g<T>(1) * wd[q + 2] + tap_g<T>(3) * wd[q + 1] + tap_g<T>(5) * wd[q];
            }
        }
    }
    if (WARP)
        __syncwarp();
    else
        __syncthreads();
    if (act) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (!INV) {
                Lp[(k0 + q) * ps] = o0[q];
                Lp[(h + k0 + q) * ps] = o1[q];
            } else {
                Lp[(2 * (k0 + q)) * ps] = o0[q];
                Lp[(2 * (k0 + q) + 1) * ps] = o1[q];
            }
        }
    }
    if (WARP)
        __syncwarp();
    else
        __syncthreads();
}

template <class T, bool INV>
__device__ __forceinline__ void dwt_pass(T* buf, int lines, int m, int ls, int ps) {
    constexpr int NT = cblk<T>();
    // lines, m and NT are powers of two; the callers keep R <= RMAX
    const int h = m >> 1;
    const int ll = __ffs(lines) - 1, lhh = __ffs(h) - 1;
    const int lnt = __ffs(NT) - 1;
    const int lruns = min(max(lnt - ll, 0), lhh);
    const int R = h >> lruns;
    const int t = threadIdx.x;
    const bool act = t < (lines << lruns);
    const int line = t & (lines - 1), k0 = (t >> ll) * R;
    T* Lp = buf + line * ls;
    switch (R) {
        case 1: dwt_run<T, INV, 1>(Lp, m, h, k0, ps, act); break;
        case 2: dwt_run<T, INV, 2>(Lp, m, h, k0, ps, act); break;
        case 4: dwt_run<T, INV, 4>(Lp, m, h, k0, ps, act); break;
        default: dwt_run<T, INV, RMAX>(Lp, m, h, k0, ps, act); break;
    }
}

// The same pass on a small block (lines * m / 2 <= 32 * RMAX pairs) by the calling warp
// alone: every lane of the warp calls it.  Each output is formed by the same expression as
// in dwt_pass, so the result is identical; only the CTA-wide barriers are gone.
template <class T, bool INV>
__device__ __forceinline__ void dwt_pass_warp(T* buf, int lines, int m, int ls, int ps) {
    const int h = m >> 1;
    const int ll = __ffs(lines) - 1, lhh = __ffs(h) - 1;
    const int lruns = min(max(5 - ll, 0), lhh);
    const int R = h >> lruns;
    const int t = threadIdx.x & 31;
    const bool act = t < (lines << lruns);
    const int line = t & (lines - 1), k0 = (t >> ll) * R;
    T* Lp = buf + line * ls;
    switch (R) {
        case 1: dwt_run<T, INV, 1, true>(Lp, m, h, k0, ps, act); break;
        case 2: dwt_run<T, INV, 2, true>(Lp, m, h, k0, ps, act); break;
        case 4: dwt_run<T, INV, 4, true>(Lp, m, h, k0, ps, act); break;
        default: dwt_run<T, INV, RMAX, true>(Lp, m, h, k0, ps, act); break;
    }
}

// Deterministic CTA sum of one double: every thread's value goes to shared memory and
// warp 0 adds them in a fixed order (few FP64 operations: GB300's FP64 rate is low).
// `scratch` holds blockDim.x doubles.
__device__ __forceinline__ double cta_sum(double v, double* scratch) {
    const int nt = blockDim.x;
    scratch[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nt; i += 32) s += scratch[i];
        s = warp_sum(s);
        if (threadIdx.x == 0) scratch[0] = s;
    }
    __syncthreads();
    const double r = scratch[0];
    __syncthreads();
    return r;
}

// Deterministic CTA sum of one float (fixed order); `scratch` holds blockDim.x floats.
__device__ __forceinline__ float cta_sumf(float v, float* scratch) {
    const int nt = blockDim.x;
    scratch[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        float s = 0.f;
        for (int i = threadIdx.x; i < nt; i += 32) s += scratch[i];
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) scratch[0] = s;
    }
    __syncthreads();
    const float r = scratch[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_t(float v) { return warp_sumf(v); }
__device__ __forceinline__ double warp_sum_t(double v) { return warp_sum(v); }
__device__ __forceinline__ float cta_sum_t(float v, double* scratch) {
    return cta_sumf(v, reinterpret_cast<float*>(scratch));
}
__device__ __forceinline__ double cta_sum_t(double v, double* scratch) { return cta_sum(v, scratch); }

// Two fixed-order CTA sums in one pass (each component in the order of cta_sum_t).
template <class T>
__device__ __forceinline__ void cta_sum2_t(T& x, T& y, double* scratch) {
    const int nt = blockDim.x;
    T* sx = reinterpret_cast<T*>(scratch);
    T* sy = sx + nt;
    sx[threadIdx.x] = x;
    sy[threadIdx.x] = y;
    __syncthreads();
    if (threadIdx.x < 32) {
        T a = T(0), b = T(0);
        for (int i = threadIdx.x; i < nt; i += 32) {
            a += sx[i];
            b += sy[i];
        }
        a = warp_sum_t(a);
        b = warp_sum_t(b);
        if (threadIdx.x == 0) {
            sx[0] = a;
            sy[0] = b;
        }
    }
    __syncthreads();
    x = sx[0];
    y = sy[0];
    __syncthreads();
}

// Levels whose block side is at most WARP_SIDE are run by warp 0 alone: a pass there is a
// few hundred cycles of barrier latency on the whole CTA and little work.
constexpr int WARP_SIDE = 16;

// The last three levels of a full decomposition (block sides 8, 4 and 2, down to the 1 x 1
// LL) as one linear map of the 8 x 8 block: the analysis is the 64 x 64 matrix A, stored
// with row stride TAIL_LD so that entry (k, o) maps input k = 8 i + j to output o; the
// synthesis is its transpose (the periodic db3 transform is orthogonal; the host checks
// that its own synthesis matches A^T).  One pass of 64 threads instead of six dependent
// level passes: each costs ~0.4 us of latency on one CTA, whatever its size.
constexpr int TAIL_LD = 65;
constexpr int TAIL_N = 64 * TAIL_LD;

// Whether the levels [lev0, levels) of a layer of side n end with the three tail levels.
__device__ __forceinline__ bool tail_applies(int n, int lev0, int levels) {
    return (n >> (levels - 1)) == 2 && levels - 3 >= lev0;
}

// y = A x (forward) or y = A^T x (inverse) on the 8 x 8 block at lbuf (stride lsd), whole
// CTA; `op` in shared memory.  Reads of x are broadcasts; reads of op are conflict-free
// (stride TAIL_LD is odd).
template <class T, bool INV>
__device__ __forceinline__ void tail_map(T* lbuf, int lsd, const T* op) {
    const int t = threadIdx.x;
    T y = T(0);
    if (t < 64) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int k = 0; k < 64; k += 4) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int kk = k + e;
                const T x = lbuf[(kk >> 3) * lsd + (kk & 7)];
                acc[e] += (INV ? op[t * TAIL_LD + kk] : op[kk * TAIL_LD + t]) * x;
            }
        }
        y = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    __syncthreads();
    if (t < 64) lbuf[(t >> 3) * lsd + (t & 7)] = y;
    __syncthreads();
}

// Forward (analysis) levels lev_begin..levels-1 of the LL block (stride lsd), whole CTA.
// `tail`: the tail operator in shared memory, or null.
template <class T>
__device__ __forceinline__ void coarse_forward(T* lbuf, const T* tail, int n, int lev_begin, int levels,
                                               int lsd) {
    const int lev_end = (tail && tail_applies(n, lev_begin, levels)) ? levels - 3 : levels;
    int lev = lev_begin;
    for (; lev < lev_end && (n >> lev) > WARP_SIDE; ++lev) {
        const int m = n >> lev;
        dwt_pass<T, false>(lbuf, m, m, lsd, 1);    // rows
        dwt_pass<T, false>(lbuf, m, m, 1, lsd);    // columns
    }
    if (lev < lev_end) {
        if (threadIdx.x < 32)
            for (; lev < lev_end; ++lev) {
                const int m = n >> lev;
                dwt_pass_warp<T, false>(lbuf, m, m, lsd, 1);
                dwt_pass_warp<T, false>(lbuf, m, m, 1, lsd);
            }
        __syncthreads();
    }
    if (lev_end < levels) tail_map<T, false>(lbuf, lsd, tail);
}

// Inverse (synthesis) levels levels-1..lev_end of the LL block.
template <class T>
__device__ __forceinline__ void coarse_inverse(T* lbuf, const T* tail, int n, int lev_end, int levels,
                                               int lsd) {
    int lev = levels - 1;
    if (tail && tail_applies(n, lev_end, levels)) {
        tail_map<T, true>(lbuf, lsd, tail);
        lev = levels - 4;
    }
    if (lev >= lev_end && (n >> lev) <= WARP_SIDE) {
        if (threadIdx.x < 32)
            for (int k = lev; k >= lev_end && (n >> k) <= WARP_SIDE; --k) {
                const int m = n >> k;
                dwt_pass_warp<T, true>(lbuf, m, m, 1, lsd);
                dwt_pass_warp<T, true>(lbuf, m, m, lsd, 1);
            }
        while (lev >= lev_end && (n >> lev) <= WARP_SIDE) --lev;
        __syncthreads();
    }
    for (; lev >= lev_end; --lev) {
        const int m = n >> lev;
        dwt_pass<T, true>(lbuf, m, m, 1, lsd);     // columns
        dwt_pass<T, true>(lbuf, m, m, lsd, 1);     // rows
    }
}

// Band of a layer owned by cluster rank r: rows (and columns) [r * rb, r * rb + rb).
__device__ __forceinline__ int band_rows(int n) { return n >= CL ? n / CL : 1; }

// Buffers of the (sensor, layer) pair terms of P and P^T, set by the host.
template <class T>
struct PairBufs {
    T* V;             // P_g,l phi_l: slot (g * n_layers + l), N+1 rows of stride vs
    T* Y;             // R^T u terms: slot (g * n_layers + l), box rows of stride box[3]
    int vs;           // row stride of a V slot
    int vslot;        // elements per V slot
    int yslot;        // elements per Y slot
    const int* box;   // per pair (g * MAXL + l): row0, rows, col0, cols
    // adjoint-projection weights per pair p = g * n_layers + l, host-built: for box column
    // (q = 0) or box row (q = 1) k, tw[((p * 2 + q) * MAXN + k) * KMAX ...] are the weights of
    // the aperture columns (rows) starting at ti[(p * 2 + q) * MAXN + k].x, .y of them
    const T* tw;
    const int2* ti;
    // staged band runs of the forward kernel, per (layer l, cluster rank r): for sensor g
    // at ((l * CL + r) * n_wfs + g) * 2, {first row, end row, col0, cols} of the band's
    // part of the term, then {offset in the stage, offset in Y, 0, 0}
    const int4* ytab;
};

// ---------------------------------------------------------------------------
// Forward layer kernel (cluster per layer).
//   SRC_NODES: y = sum_g P_g^T u_g (Sec. 2, adjoint), then W y;  SRC_PHI: W phi.
//   DST_COEF:  write W y (b of Sec. 3.1 when u comes from the measured slopes);
//   DST_APPLY: write q = W y + alpha D p and p.q (Eq. 6); the grid's last CTA forms
//              the total p.q in a fixed order.
// P_g^T is separable, y = R_y^T u R_x: for each sensor, pass X contracts the staged node
// rows with the column weights, pass Y with the row weights.  The sensors' node rows and
// tables are staged with cp.async in a double buffer, one sensor ahead of the compute.
// ---------------------------------------------------------------------------
template <class T>
struct ClArgs {
    const T* in;        // u (nodes), phi, or coefficients
    const T* pin;       // p of the apply
    T* out;
    T* pupd;            // p advanced in place (inverse kernel with update)
    const T* zupd;
    PcgSlots pcg;
    int iter;           // p.q slot of the apply / CG iteration of the update
    int zero_piston;    // data term of M: forward kernel, the full-depth LL output is exactly
                        // 0; inverse kernel, the full-depth LL input is left out
    // augmented direction update (inverse kernel, PUPD = 2): output p_new, the previous
    // frame's directions P_j (stride aug_ld, aug_m of them), q_j.z at aug_tot[AUG_MAX + j]
    // and p_j.q_j at aug_pq[j]
    T* pout;
    const T* augP;
    const double* aug_tot;
    const double* aug_pq;
    long long aug_ld;
    int aug_m;
    // deferred q_j.z totals (aug_pcnt > 0): dot j's shares at aug_parts + j * aug_pcnt, totalled
    // here in the fixed order instead of read from aug_tot
    const double* aug_parts;
    int aug_pcnt;
    // the initial residual's vector step fused into the forward kernel (DST_APPLY_INIT): the
    // vectors r, z, p, b, b_prev, J^-1; r.z shares at rzp[l * CL + rank], total into rz slot
    // rzslot
    T* vr;
    T* vz;
    T* vp;
    const T* vb;
    T* vbprev;
    const T* vj;
    double* rzp;
    int rzslot;
    // Deferred totals.  defer_total (forward kernel): the CTA shares of p.q (APPLY) or r.z
    // (APPLY_INIT) are stored and the total is left to the next kernel that needs it, so no
    // CTA waits for a grid-wide arrival count.  rz_cnt > 0 (inverse kernel): the r.z total
    // of slot rz_slot is formed from the rz_cnt shares at rz_parts (fixed order, the same in
    // every CTA), used for beta, and stored by the first CTA.
    int defer_total;
    const double* rz_parts;
    int rz_cnt;
    int rz_slot;
};

struct ClLayout {       // shared-memory offsets set by the host, in T units
    int ybuf, cbuf, lbuf, stage, stage2, tbuf;
    int tail;           // the tail operator (TAIL_N), staged by the leader; 0 = none
    int total;
    int umax;           // one staging buffer of the P^T pipeline
    int ystg;           // staged pair terms of the band (forward kernel), 0 = not staged
    int ydirect;        // the band's pair terms read straight from L2 in 16-byte groups
    int lstage;         // the LL quadrant's epilogue operands, staged by the leader (3 x
                        // (MAXN / 2)^2); 0 = the LL epilogue is shared out over the cluster
};

constexpr int KMAX = 8;      // aperture rows / columns touching one layer row / column

// Body of the forward layer kernel for layer l; `ctas` = CTAs of the instance's grid
// (the p.q total is formed by the last of them to arrive).
template <class T, int SRC, int DST>
__device__ __forceinline__ void cl_fwd_body(const Desc<T>& d, const ClArgs<T>& a, const ClLayout& lay,
                                            const PairBufs<T>& pb, const int l, const unsigned ctas) {
    constexpr int NT = cblk<T>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);            // RED_DBL doubles
    T* sm = reinterpret_cast<T*>(red + RED_DBL);
    __shared__ bool last;
    cg::cluster_group cluster = cg::this_cluster();
    const int r = static_cast<int>(cluster.block_rank());
    const LayerInfo L = d.L[l];
    const int n = L.n, off = L.off, h = n >> 1;
    const int rb = band_rows(n);
    const int lrb = L.log2n >= 3 ? L.log2n - 3 : 0;   // log2(rb), CL = 8
    const int lh = L.log2n - 1;                        // log2(n / 2)
    const int r0 = r * rb;
    const bool has_band = r0 < n;
    const bool coarse = L.levels >= 2;
    T* ybuf = sm + lay.ybuf;          // rb x (n + 1)
    T* cbuf = sm + lay.cbuf;          // n x (rb + 1)
    T* lbuf = sm + lay.lbuf;          // h x (h + 1)
    const int ys = n + 1, cs = rb + 1, lsd = h + 1;

    // the exchanges below push into peers' shared memory before the first full cluster
    // barrier: arrive now, wait before the first push, so that every CTA has started
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
    // the tail operator of the leader's coarse levels (constant data: staged at once; every
    // band path below waits for its copies before the first cluster barrier)
    const bool tail_on = coarse && r == 0 && lay.tail > 0 && d.tailop != nullptr;
    if (tail_on) stage16(sm + lay.tail, d.tailop, TAIL_N, threadIdx.x, NT);
    // ---- 0. prefetch the epilogue operands of the column band (independent of u) ----
    constexpr int PF = MAXN * (MAXN / CL) / NT;     // column-band positions per thread
    const int row_start = (coarse && r0 < h) ? h : 0;
    const int ecnt = has_band ? (n - row_start) * rb : 0;
    T pre_p[PF];
    // D is one value per (layer, level) (Sec. 3.1): the layer's row of the table, in shared
    // memory, indexed by the level of each position
    __shared__ T sD[MAXLEV + 1];
    if (threadIdx.x <= MAXLEV) sD[threadIdx.x] = d.Dlev[l][threadIdx.x];
    // the band-run table of the staged sum, loaded now so that its latency overlaps
    int4 ytv = make_int4(0, 0, 0, 0);
    if (SRC == LSRC_NODES && (lay.ystg > 0 || lay.ydirect) && has_band && threadIdx.x < 2 * d.n_wfs)
        ytv = pb.ytab[(l * CL + r) * 2 * d.n_wfs + threadIdx.x];
    // this CTA's share of the LL quadrant's rows (coarse layers): [lr0, lr1), hb rows each.
    // A quadrant narrower than 32 stays with the leader: sharing it out costs a cluster
    // barrier, more than the leader's few positions take.
    constexpr bool INIT = DST == LDST_APPLY_INIT || DST == LDST_RESID_INIT;   // fused r0 step
    constexpr bool NEEDB = DST == LDST_APPLY_INIT;                              // b read
    constexpr bool QAPPLY = DST == LDST_APPLY || INIT;                         // p read
    constexpr int PL = ((MAXN / 2) * (MAXN / 2) / CL + NT - 1) / NT;   // LL-share positions per thread
    // With lay.lstage (single precision), the leader stages the LL quadrant's operands in
    // shared memory now and forms the whole LL epilogue itself after its coarse levels: no
    // rows go back to the other ranks and no third cluster barrier is needed.
    const bool lstaged = lay.lstage > 0 && coarse;
    const bool ldist = !lstaged && h >= 32;
    const int hb = ldist ? h >> 3 : h;
    const int lr0 = coarse ? min(r * hb, h) : 0, lr1 = coarse ? min(lr0 + hb, h) : 0;
    const int lcnt = lstaged ? 0 : (lr1 - lr0) * h;     // LL positions prefetched to registers
    T* lsp = sm + lay.lstage;                           // staged p, b, J^-1 of LL (stride h)
    T* lsb = lsp + (MAXN / 2) * (MAXN / 2);
    T* lsj = lsb + (MAXN / 2) * (MAXN / 2);
    if (lstaged && r == 0 && QAPPLY) {
        constexpr int V = vec16<T>();
        const int lc = lh - (V == 4 ? 2 : 1);           // log2 of the 16-byte chunks per row
        for (int k = threadIdx.x; k < (h << lc); k += NT) {
            const int i = k >> lc, c = (k & ((1 << lc) - 1)) * V, pos = off + i * n + c;
            cp_async16(lsp + i * h + c, a.pin + pos);
            if (NEEDB) cp_async16(lsb + i * h + c, a.vb + pos);
            if (INIT) cp_async16(lsj + i * h + c, a.vj + pos);
        }
    }
    // operands of the epilogue at this CTA's positions (band, then LL share), loaded now so
    // that their latency overlaps: p; with the fused initial residual also b and J^-1
    T pl[PL], xb[PF], xl[PL], jb[PF], jl[PL];
    if (QAPPLY) {
#pragma unroll
        for (int s = 0; s < PF; ++s) {
            const int k = threadIdx.x + s * NT;
            if (k < ecnt) {
                const int pos = off + (row_start + (k >> lrb)) * n + r0 + (k & (rb - 1));
                pre_p[s] = a.pin[pos];
                if (NEEDB) xb[s] = a.vb[pos];
                if (INIT) jb[s] = a.vj[pos];
            }
        }
#pragma unroll
        for (int s = 0; s < PL; ++s) {
            const int k = threadIdx.x + s * NT;
            if (k < lcnt) {
                const int pos = off + (lr0 + (k >> lh)) * n + (k & (h - 1));
                pl[s] = a.pin[pos];
                if (NEEDB) xl[s] = a.vb[pos];
                if (INIT) jl[s] = a.vj[pos];
            }
        }
    }

    // Everything above reads only data that the kernel two launches back (or earlier) had
    // written: p and b are inputs of the apply, written before its first kernel.  The band
    // below reads the adjoint projection's output, written by the previous kernel.
    pdl_wait();
    // ---- 1. the row band of y ---------------------------------------------------
    if (has_band) {
        if (SRC == LSRC_PHI) {
            for (int k = threadIdx.x; k < rb * n; k += NT) {
                const int i = (k >> L.log2n), j = k - i * n;
                cp_async(ybuf + i * ys + j, a.in + off + (r0 + i) * n + j);
            }
            cp_async_wait();
            __syncthreads();
        } else if (lay.ydirect) {
            // y = sum_g R_y,gl^T u_g R_x,gl over this band, read straight from the pair slots:
            // the boxes' columns are 16-byte groups of the layer grid (host-checked), so a
            // thread owns one group and issues one 16-byte L2 read per sensor, all in flight
            // together (single precision: one group per thread), then adds them in the fixed
            // sensor order.  The runs of the band (host table) give each sensor's rows.
            constexpr int V = vec16<T>();
            using VT = typename Vec16<T>::type;
            __shared__ int4 ygb[MAXG];        // per sensor: first and end band row, col0, cols
            __shared__ int4 ygx[MAXG];        // per sensor: offset in the stage, offset in Y
            if (threadIdx.x < 2 * d.n_wfs) {
                if (threadIdx.x & 1)
                    ygx[threadIdx.x >> 1] = ytv;
                else
                    ygb[threadIdx.x >> 1] = ytv;
            }
            __syncthreads();
            const int lg = L.log2n - (V == 4 ? 2 : 1);        // log2 of the groups per row
            for (int grp = threadIdx.x; grp < (rb << lg); grp += NT) {
                const int ii = grp >> lg, j0 = (grp & ((1 << lg) - 1)) * V, i = r0 + ii;
                VT v[MAXG];
                bool in[MAXG];
#pragma unroll
                for (int g = 0; g < MAXG; ++g) {
                    in[g] = false;
                    if (g < d.n_wfs) {
                        const int4 bx = ygb[g];
                        in[g] = i >= bx.x && i < bx.y && j0 >= bx.z && j0 < bx.z + bx.w;
                        if (in[g])
                            v[g] = __ldcg(reinterpret_cast<const VT*>(pb.Y + ygx[g].y + (i - bx.x) * bx.w +
                                                                      (j0 - bx.z)));
                    }
                }
                T acc[V];
#pragma unroll
                for (int e = 0; e < V; ++e) acc[e] = T(0);
#pragma unroll
                for (int g = 0; g < MAXG; ++g)
                    if (in[g]) {
#pragma unroll
                        for (int e = 0; e < V; ++e) acc[e] += Vec16<T>::at(v[g], e);
                    }
#pragma unroll
                for (int e = 0; e < V; ++e) ybuf[ii * ys + j0 + e] = acc[e];
            }
            cp_async_wait();
            __syncthreads();
        } else if (lay.ystg > 0) {
            // y = sum_g R_y,gl^T u_g R_x,gl over this band.  The band's rows of sensor g's
            // term are one contiguous run of its pair slot (rows of box[g][l][3] columns);
            // the runs (host table) are staged with 16-byte copies, all in flight together,
            // and added from shared memory in the fixed sensor order.  The boxes' columns
            // are 16-byte groups of the layer grid (host-checked), so a thread adds whole
            // groups: one 16-byte shared-memory read per sensor and group.
            constexpr int V = vec16<T>();
            using VT = typename Vec16<T>::type;
            constexpr int KG = (MAXN * (MAXN / CL) / V + NT - 1) / NT;   // groups per thread
            __shared__ int4 ygb[MAXG];        // per sensor: first and end band row, col0, cols
            __shared__ int4 ygx[MAXG];        // per sensor: offset in the stage, offset in Y
            T* ystg = sm + lay.ystg;
            if (threadIdx.x < 2 * d.n_wfs) {
                if (threadIdx.x & 1)
                    ygx[threadIdx.x >> 1] = ytv;
                else
                    ygb[threadIdx.x >> 1] = ytv;
            }
            __syncthreads();
            for (int g = 0; g < d.n_wfs; ++g) {
                const int4 bx = ygb[g];
                if (bx.y > bx.x) stage16(ystg + ygx[g].x, pb.Y + ygx[g].y, (bx.y - bx.x) * bx.w, threadIdx.x, NT);
            }
            const int lg = L.log2n - (V == 4 ? 2 : 1);        // log2 of the groups per row
            const int ngrp = rb << lg;
            cp_async_wait();
            __syncthreads();
#pragma unroll
            for (int s2 = 0; s2 < KG; ++s2) {
                const int grp = threadIdx.x + s2 * NT;
                if (grp < ngrp) {
                    const int ii = grp >> lg, j0 = (grp & ((1 << lg) - 1)) * V, i = r0 + ii;
                    T acc[V];
#pragma unroll
                    for (int e = 0; e < V; ++e) acc[e] = T(0);
                    for (int g = 0; g < d.n_wfs; ++g) {
                        const int4 bx = ygb[g];
                        if (i >= bx.x && i < bx.y && j0 >= bx.z && j0 < bx.z + bx.w) {
                            const VT v = *reinterpret_cast<const VT*>(ystg + ygx[g].x + (i - bx.x) * bx.w + (j0 - bx.z));
#pragma unroll
                            for (int e = 0; e < V; ++e) acc[e] += Vec16<T>::at(v, e);
                        }
                    }
#pragma unroll
                    for (int e = 0; e < V; ++e) ybuf[ii * ys + j0 + e] = acc[e];
                }
            }
            __syncthreads();
        } else {
            // y = sum_g R_y,gl^T u_g R_x,gl: add the pair terms (fixed sensor order) over
            // this band; a term is zero outside its footprint box
            // every load is issued unconditionally from a clamped index, then masked, so
            // that the sensors' loads are in flight together
            for (int k = threadIdx.x; k < rb * n; k += NT) {
                const int ii = k >> L.log2n, j = k & (n - 1), i = r0 + ii;
                T v[MAXG];
                bool in[MAXG];
#pragma unroll
                for (int g = 0; g < MAXG; ++g) {
                    in[g] = false;
                    if (g < d.n_wfs) {
                        const int ri = i - d.box[g][l][0], cj = j - d.box[g][l][2];
                        in[g] = ri >= 0 && ri < d.box[g][l][1] && cj >= 0 && cj < d.box[g][l][3];
                        const int rc = min(max(ri, 0), d.box[g][l][1] - 1);
                        const int cc = min(max(cj, 0), d.box[g][l][3] - 1);
                        v[g] = pb.Y[(g * d.n_layers + l) * pb.yslot + rc * d.box[g][l][3] + cc];
                    }
                }
                T acc = T(0);
#pragma unroll
                for (int g = 0; g < MAXG; ++g)
                    if (in[g]) acc += v[g];
                ybuf[ii * ys + j] = acc;
            }
            cp_async_wait();
            __syncthreads();
        }
        // ---- 2. level-0 analysis along the rows of the band --------------------
        dwt_pass<T, false>(ybuf, rb, n, ys, 1);
    }
    asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");
    // ---- 3. the band's rows go to every column band's owner (pushed), column analysis ---
    if (has_band) {
        for (int k = threadIdx.x; k < rb * n; k += NT) {
            const int ii = k >> L.log2n, j = k & (n - 1);
            cluster.map_shared_rank(cbuf, static_cast<unsigned>(j >> lrb))[(r0 + ii) * cs + (j & (rb - 1))] =
                ybuf[ii * ys + j];
        }
    }
    cluster.sync();                                                       // #1: column tiles complete
    DotAcc<T> dot;                 // p.q share of this CTA (double accuracy)
    DotAcc<T> drz;                 // r.z share (fused initial residual)
    // The epilogue at one position: v = (W y)(i, j), p and the prefetched operands.
    //   APPLY: q = v + alpha D p, written, p.q;  COEF: v written;
    //   APPLY_INIT (initial residual, Algorithm 1): r = b - q, z = J^-1 r, p = z, b_prev = b, r.z.
    auto epi = [&](int i, int j, int pos, T v, T p, T x, T jv) {
        if (!QAPPLY) {
            a.out[pos] = v;
            return;
        }
        if (DST == LDST_RESID_INIT) {
            // v is the residual's data term: r0 = v - alpha D c0
            const T rr = v - d.alpha * sD[level_of(i, j, L)] * p;
            const T z = jv * rr;
            a.vr[pos] = rr;
            a.vz[pos] = z;
            a.vp[pos] = z;
            drz.add(rr, z);
            return;
        }
        const T q = v + d.alpha * sD[level_of(i, j, L)] * p;
        if (DST == LDST_APPLY) {
            a.out[pos] = q;
            dot.add(p, q);
        } else {
            const T rr = x - q;
            const T z = jv * rr;
            a.vr[pos] = rr;
            a.vz[pos] = z;
            a.vp[pos] = z;
            a.vbprev[pos] = x;
            drz.add(rr, z);
        }
    };
    if (has_band) {
        dwt_pass<T, false>(cbuf, rb, n, 1, cs);
        // ---- 4. the LL quadrant's part of this column band goes to the leader (pushed) ---
        if (coarse && r0 < h) {
            T* lead = cluster.map_shared_rank(lbuf, 0);
            for (int k = threadIdx.x; k < h * rb; k += NT) {
                const int i = k >> lrb, jj = k & (rb - 1);
                lead[i * lsd + r0 + jj] = cbuf[i * cs + jj];
            }
        }
        // ---- 5. epilogue of the column band (below the LL quadrant when coarse), while the
        // leader's coarse levels wait for the barrier -----------------------------------------
        if (!coarse && a.zero_piston && L.full && r == 0 && threadIdx.x == 0) cbuf[0] = T(0);
        __syncthreads();
#pragma unroll
        for (int s2 = 0; s2 < PF; ++s2) {
            const int k = threadIdx.x + s2 * NT;
            if (k < ecnt) {
                const int i = row_start + (k >> lrb), jj = (k & (rb - 1));
                epi(i, r0 + jj, off + i * n + r0 + jj, cbuf[i * cs + jj], pre_p[s2], xb[s2], jb[s2]);
            }
        }
    }
    cluster.sync();                                                       // #2: the leader holds LL
    pdl_trigger();
    if (coarse) {
        // ---- 6. the leader's coarse levels; the LL quadrant's rows go back to their
        // owners (pushed), whose epilogue takes its share of them ----------------------------
        if (r == 0) {
            coarse_forward<T>(lbuf, tail_on ? sm + lay.tail : nullptr, n, 1, L.levels, lsd);
            // The data term has no piston component: Gamma annihilates constants and bilinear
            // weights sum to one, so its full-depth LL coefficient is exactly 0.  Write that
            // zero rather than the rounding residue of a cancelling sum, which the solve would
            // amplify by 1 / (alpha D_LL).
            if (a.zero_piston && L.full && threadIdx.x == 0) lbuf[0] = T(0);
            __syncthreads();
            if (ldist)
                for (int k = threadIdx.x; k < h * h; k += NT) {
                    const int i = k >> lh, j = k & (h - 1), q = i / hb;
                    cluster.map_shared_rank(ybuf, static_cast<unsigned>(q))[(i - q * hb) * h + j] =
                        lbuf[i * lsd + j];
                }
        }
        if (ldist) cluster.sync();                                        // #3: no remote access after this
        if (lstaged) {
            if (r == 0)
                for (int k = threadIdx.x; k < h * h; k += NT) {
                    const int i = k >> lh, j = k & (h - 1);
                    epi(i, j, off + i * n + j, lbuf[i * lsd + j], QAPPLY ? lsp[k] : T(0),
                        NEEDB ? lsb[k] : T(0), INIT ? lsj[k] : T(0));
                }
        } else {
#pragma unroll
            for (int s2 = 0; s2 < PL; ++s2) {
                const int k = threadIdx.x + s2 * NT;
                if (k < lcnt) {
                    const int i = lr0 + (k >> lh), j = k & (h - 1);
                    epi(i, j, off + i * n + j, ldist ? ybuf[k] : lbuf[i * lsd + j], pl[s2], xl[s2], jl[s2]);
                }
            }
        }
    }
    if (DST == LDST_APPLY) {
        double* slots = a.pcg.pqpart + a.iter * PQ_SLOTS;
        cta_dot_store(dot, red, slots + l * CL + r);
        if (!a.defer_total && last_arrival(a.pcg.count + 1, ctas, &last) && threadIdx.x < 32) {
            // fixed order: layer-major, rank-minor over the slots of the layers present
            const double tot = warp_total(slots, d.n_layers * CL, &dot);
            if (threadIdx.x == 0) {
                a.pcg.pqtot[a.iter] = tot;
                a.pcg.count[1] = 0;
            }
        }
    }
    if (INIT) {
        // r.z of the new residual into rz slot `rzslot`, fixed order over the layer CTAs
        cta_dot_store(drz, red, a.rzp + l * CL + r);
        if (!a.defer_total && last_arrival(a.pcg.count, ctas, &last) && threadIdx.x < 32) {
            const double tot = warp_total(a.rzp, d.n_layers * CL, &drz);
            if (threadIdx.x == 0) {
                a.pcg.rztot[a.rzslot] = tot;
                a.pcg.count[0] = 0;
            }
        }
    }
}

template <class T, int SRC, int DST>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(cblk<T>(), 1)
    k_cl_fwd(__grid_constant__ const Desc<T> d, __grid_constant__ const ClArgs<T> a,
             __grid_constant__ const ClLayout lay, __grid_constant__ const PairBufs<T> pb) {
    cl_fwd_body<T, SRC, DST>(d, a, lay, pb, blockIdx.y, gridDim.x * gridDim.y);
}

// ---------------------------------------------------------------------------
// Inverse layer kernel (cluster per layer): phi = W^T c, optionally advancing the CG
// direction first (Sec. 3.3).  PUPD = 0: phi = W^T a.in.  PUPD = 1: p = z + beta p in place
// (a.pupd), beta = rz_k / rz_(k-1), then phi = W^T p.  PUPD = 2, the augmented PCG of
// Sec. 3.4: p_new = z + beta p_old - sum_j mu_j P_j into a.pout, mu_j = q_j.z / p_j.q_j of
// the previous frame's directions P_j (p_old = a.pupd; none, and beta = 0, for a frame's
// first direction), then phi = W^T p_new.  The direction update is spread over the
// cluster: every CTA updates its column band (below the LL quadrant when coarse) and a
// share of the LL quadrant's rows, which it pushes to the leader for the coarse levels.
// ---------------------------------------------------------------------------
template <class T, int PUPD>
__device__ __forceinline__ void cl_inv_body(const Desc<T>& d, const ClArgs<T>& a, const ClLayout& lay,
                                            const int l) {
    constexpr int NT = cblk<T>();
    constexpr int PF = MAXN * (MAXN / CL) / NT;                      // band positions per thread
    constexpr int PL = ((MAXN / 2) * (MAXN / 2) / CL + NT - 1) / NT; // LL-share positions per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);
    T* sm = reinterpret_cast<T*>(red + RED_DBL);
    cg::cluster_group cluster = cg::this_cluster();
    const int r = static_cast<int>(cluster.block_rank());
    const LayerInfo L = d.L[l];
    const int n = L.n, off = L.off, h = n >> 1;
    const int rb = band_rows(n);
    const int lrb = L.log2n >= 3 ? L.log2n - 3 : 0;   // log2(rb), CL = 8
    const int lh = L.log2n - 1;                        // log2(n / 2)
    const int r0 = r * rb;
    const bool has_band = r0 < n;
    T* ybuf = sm + lay.ybuf;
    T* cbuf = sm + lay.cbuf;
    T* lbuf = sm + lay.lbuf;
    const int ys = n + 1, cs = rb + 1, lsd = h + 1;
    const bool coarse = L.levels >= 2;
    // this CTA's rows of the LL quadrant (coarse layers): [lr0, lr1); a quadrant narrower
    // than 32 stays with the leader, as in the forward kernel
    const bool ldist = h >= 32;
    const int hb = ldist ? h >> 3 : h;                 // h / CL
    const int lr0 = coarse ? min(r * hb, h) : 0, lr1 = coarse ? min(lr0 + hb, h) : 0;
    const int lcnt = (lr1 - lr0) * h;

    // beta = rz_k / rz_(k-1) and the mu_j, formed once (an FP64 division costs ~10 FP64
    // instructions, and GB300 issues a warp's FP64 instruction in ~64 cycles) and broadcast
    __shared__ T sbeta;
    __shared__ T smu[AUG_MAX];
    const bool has_old = PUPD == 1 || (PUPD == 2 && a.pupd != nullptr);
    const bool stage_src = PUPD == 0 || has_old;
    const T* src = PUPD ? a.pupd : a.in;
    T* pdst = PUPD == 2 ? a.pout : a.pupd;
    // the exchanges below push into peers' shared memory before the first full cluster
    // barrier: arrive now, wait before the first push, so that every CTA has started
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
    // ---- 1. stage this CTA's coefficients: its column band and its LL rows.  Rows go
    // through unpadded staging tiles in 16-byte chunks when aligned.
    constexpr int V = vec16<T>();
    const int row_start = (coarse && r0 < h) ? h : 0;
    const int nrow = n - row_start;
    T* sp = sm + lay.stage;                     // column band, stride rb: p (or c)
    T* sz = sp + MAXN * (MAXN / CL);            // column band: z (PUPD)
    T* lp = sm + lay.stage2;                    // LL rows, stride h: p (or c)
    T* lz = lp + (MAXN / 2) * (MAXN / 2);       // LL rows: z (PUPD)
    // the tail operator of the leader's coarse levels, with the staging copies below
    const bool tail_on = coarse && r == 0 && lay.tail > 0 && d.tailop != nullptr;
    if (tail_on) stage16(sm + lay.tail, d.tailop, TAIL_N, threadIdx.x, NT);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = NT >> 5;
    // The copies of one vector (x = p or c, or z): the column band, then the LL rows.
    auto stage_vec = [&](const T* x, T* dst_band, T* dst_ll) {
        if (has_band) {
            if ((rb & (V - 1)) == 0) {
                const int cpr = rb / V;             // chunks per row (a power of two)
                const int lcpr = __ffs(cpr) - 1;
                for (int k = threadIdx.x; k < nrow * cpr; k += NT) {
                    const int i = k >> lcpr, c = k & (cpr - 1);
                    cp_async16(dst_band + i * rb + c * V, x + off + (row_start + i) * n + r0 + c * V);
                }
            } else {
                for (int k = threadIdx.x; k < nrow * rb; k += NT) {
                    const int i = k >> lrb, jj = k & (rb - 1);
                    cp_async(dst_band + k, x + off + (row_start + i) * n + r0 + jj);
                }
            }
        }
        for (int i = lr0 + warp; i < lr1; i += nwarp) {
            const T* xs = x + off + i * n;
            T* dl = dst_ll + (i - lr0) * h;
            if ((h & (V - 1)) == 0) {
                for (int c = lane; c < h / V; c += 32) cp_async16(dl + c * V, xs + c * V);
            } else {
                for (int j = lane; j < h; j += 32) cp_async(dl + j, xs + j);
            }
        }
    };
    // The direction being advanced (PUPD > 0: p_old, last written by the inverse kernel of
    // the previous iteration) is staged before the dependency wait; z, the plain input (its
    // writer may be the previous kernel) and the scalars after it.
    if (PUPD && stage_src) stage_vec(src, sp, lp);
    pdl_wait();
    if (!PUPD && stage_src) stage_vec(src, sp, lp);
    if (PUPD) stage_vec(a.zupd, sz, lz);
    // beta and mu are formed while the copies are in flight; a deferred r.z total first
    // (warp 0, fixed order: the same value in every CTA)
    if (threadIdx.x < 32 && (PUPD || a.rz_cnt > 0)) {
        double rz_new = 0.0;
        if (a.rz_cnt > 0) {
            rz_new = warp_total(a.rz_parts, a.rz_cnt, static_cast<const DotAcc<T>*>(nullptr));
            if (threadIdx.x == 0 && l == 0 && r == 0) a.pcg.rztot[a.rz_slot] = rz_new;
        }
        if (PUPD && threadIdx.x == 0) {
            double b = 0.0;
            if (has_old) {
                if (a.rz_cnt == 0) rz_new = a.pcg.rztot[a.iter];
                const double rz_old = a.pcg.rztot[a.iter - 1];
                b = rz_old != 0.0 ? rz_new / rz_old : 0.0;
            }
            sbeta = T(b);
        }
    }
    if (PUPD == 2) {
        if (a.aug_pcnt > 0) {
            // deferred totals: warps 1, 2, ... each total dot j in the fixed order
            const int warp1 = threadIdx.x >> 5, nw1 = NT >> 5;
            for (int j = warp1 - 1; warp1 > 0 && j < a.aug_m; j += nw1 - 1) {
                const double num = warp_total(a.aug_parts + static_cast<long long>(j) * a.aug_pcnt, a.aug_pcnt,
                                              static_cast<const DotAcc<T>*>(nullptr));
                if ((threadIdx.x & 31) == 0) {
                    const double den = a.aug_pq[j];
                    smu[j] = T(den > 0.0 ? num / den : 0.0);
                }
            }
        } else if (threadIdx.x >= 32 && threadIdx.x < 32 + a.aug_m) {
            const int j = threadIdx.x - 32;
            const double num = a.aug_tot[AUG_MAX + j], den = a.aug_pq[j];
            smu[j] = T(den > 0.0 ? num / den : 0.0);
        }
    }
    // the augmented update's sum_j mu_j P_j at this thread's positions, its loads in flight
    // beside the staging copies
    T cb[PF], cl[PL];
#pragma unroll
    for (int s2 = 0; s2 < PF; ++s2) cb[s2] = T(0);
#pragma unroll
    for (int s2 = 0; s2 < PL; ++s2) cl[s2] = T(0);
    if (PUPD == 2) {
        __syncthreads();                                             // smu
        for (int j = 0; j < a.aug_m; ++j) {
            const T mu = smu[j];
            const T* Pj = a.augP + static_cast<long long>(j) * a.aug_ld + off;
#pragma unroll
            for (int s2 = 0; s2 < PF; ++s2) {
                const int k = threadIdx.x + s2 * NT;
                if (has_band && k < nrow * rb)
                    cb[s2] += mu * __ldg(Pj + (row_start + (k >> lrb)) * n + r0 + (k & (rb - 1)));
            }
#pragma unroll
            for (int s2 = 0; s2 < PL; ++s2) {
                const int k = threadIdx.x + s2 * NT;
                if (k < lcnt) cl[s2] += mu * __ldg(Pj + (lr0 + (k >> lh)) * n + (k & (h - 1)));
            }
        }
    }
    cp_async_wait();
    __syncthreads();
    const T beta = PUPD ? sbeta : T(0);
    // the direction update into the padded tiles and back to global
#pragma unroll
    for (int s2 = 0; s2 < PF; ++s2) {
        const int k = threadIdx.x + s2 * NT;
        if (has_band && k < nrow * rb) {
            const int i = k >> lrb, jj = k & (rb - 1);
            T p = stage_src ? sp[k] : T(0);
            if (PUPD == 1) p = sz[k] + beta * p;
            if (PUPD == 2) p = (has_old ? sz[k] + beta * p : sz[k]) - cb[s2];
            if (PUPD) pdst[off + (row_start + i) * n + r0 + jj] = p;
            cbuf[(row_start + i) * cs + jj] = p;
        }
    }
#pragma unroll
    for (int s2 = 0; s2 < PL; ++s2) {
        const int k = threadIdx.x + s2 * NT;
        if (k < lcnt) {
            T p = stage_src ? lp[k] : T(0);
            if (PUPD == 1) p = lz[k] + beta * p;
            if (PUPD == 2) p = (has_old ? lz[k] + beta * p : lz[k]) - cl[s2];
            if (PUPD) pdst[off + (lr0 + (k >> lh)) * n + (k & (h - 1))] = p;
            lp[k] = p;
        }
    }
    // Input of the data path of M (a.zero_piston): Gamma annihilates constants and bilinear
    // weights sum to one, so a full-depth layer's piston coefficient (its constant function)
    // contributes nothing to P, Gamma and back, and is left out.  Exact; without it a large
    // piston component (the adjoint vectors of the gradient passes carry one, J^-1 of that
    // coefficient being ~1e5) rounds into phi and leaks through the differences of Gamma.
    // Element (0, 0) was filled by thread 0 of rank 0; p itself is stored unchanged.
    if (a.zero_piston && L.full && r == 0 && threadIdx.x == 0) {
        if (coarse)
            lp[0] = T(0);
        else
            cbuf[0] = T(0);
    }
    __syncthreads();
    asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");
    // ---- 2. the LL rows go to the leader (pushed); the leader synthesises the coarse
    // levels and pushes the quadrant's columns into the column bands' tiles --------------
    if (coarse) {
        T* lead = ldist ? cluster.map_shared_rank(lbuf, 0) : lbuf;
        for (int k = threadIdx.x; k < lcnt; k += NT) lead[(lr0 + (k >> lh)) * lsd + (k & (h - 1))] = lp[k];
        if (ldist)
            cluster.sync();                                               // #0: the leader holds LL
        else
            __syncthreads();
        if (r == 0) {
            coarse_inverse<T>(lbuf, tail_on ? sm + lay.tail : nullptr, n, 1, L.levels, lsd);
            for (int k = threadIdx.x; k < h * h; k += NT) {
                const int i = k >> lh, j = k & (h - 1);
                cluster.map_shared_rank(cbuf, static_cast<unsigned>(j >> lrb))[i * cs + (j & (rb - 1))] =
                    lbuf[i * lsd + j];
            }
        }
    }
    cluster.sync();                                                       // #1
    pdl_trigger();
    // ---- 3. column synthesis of level 0 on the column band; its rows go to every row
    // band's owner (pushed) -----------------------------------------------------------------
    if (has_band) {
        dwt_pass<T, true>(cbuf, rb, n, 1, cs);
        for (int k = threadIdx.x; k < n * rb; k += NT) {
            const int i = k >> lrb, jj = k & (rb - 1), q = i >> lrb;
            cluster.map_shared_rank(ybuf, static_cast<unsigned>(q))[(i - q * rb) * ys + r0 + jj] = cbuf[i * cs + jj];
        }
    }
    cluster.sync();                                                       // #2: no remote access after this
    // ---- 4. row synthesis of the row band, store phi --------------------------------------
    if (has_band) {
        dwt_pass<T, true>(ybuf, rb, n, ys, 1);
        for (int k = threadIdx.x; k < rb * n; k += NT) {
            const int ii = (k >> L.log2n), j = k - ii * n;
            a.out[off + (r0 + ii) * n + j] = ybuf[ii * ys + j];
        }
    }
}

template <class T, int PUPD>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(cblk<T>(), 1)
    k_cl_inv(__grid_constant__ const Desc<T> d, __grid_constant__ const ClArgs<T> a,
             __grid_constant__ const ClLayout lay) {
    cl_inv_body<T, PUPD>(d, a, lay, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Sensor kernel (cluster per sensor): P_g (Sec. 2), Gamma_g, C_hat_g^-1 (Eq. 2, Sec. 3.2)
// and Gamma_g^T, each CTA on a band of subaperture rows.  SRC_PHI: slopes of the
// projected layers (the M-apply); SRC_SLOPES: measured slopes (the right-hand side).
// ---------------------------------------------------------------------------
struct SensorLayout {
    int phsub, V, SX, SY, halo, total;         // T units
    int msk;            // the band's rows of the active-subaperture index table (ints)
};

template <class T, int SRC>
__device__ __forceinline__ void cl_sensor_body(const Desc<T>& d, const SensorArgs<T>& a,
                                               const SensorLayout& lay, const PairBufs<T>& pb,
                                               const int g) {
    constexpr int NT = cblk<T>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);                 // 2*CWMAX + 8
    double* part = red + RED_DBL;                                 // 2 + 2*MAXCOARSE
    int* tab = reinterpret_cast<int*>(part + 2 + 2 * MAXCOARSE);       // 4 * MAXL + 4 ints
    T* sm = reinterpret_cast<T*>(tab + 4 * MAXL + 4);
    cg::cluster_group cluster = cg::this_cluster();
    const int r = static_cast<int>(cluster.block_rank());
    const WfsInfo W = d.G[g];
    const int N = W.N, NP = N + 1;
    const int sr = (N + CL - 1) / CL;
    const int s0 = r * sr < N ? r * sr : N;
    const int s1 = (r + 1) * sr < N ? (r + 1) * sr : N;
    const int rows = s1 - s0;                  // subaperture rows of this CTA (may be 0)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = NT >> 5;
    const int* sidx = d.sidx + W.mask_off;
    const T inv = T(W.sig2inv);
    const T nbinv = T(1) / T(W.nb);
    T* V = sm + lay.V;          // (rows + 1) x NP
    T* SX = sm + lay.SX;        // rows x N
    T* SY = sm + lay.SY;
    T* halo = sm + lay.halo;    // 2 x N: weighted slopes of subaperture row s0 - 1
    T* cw = halo + 2 * N;       // 2 x MAXCOARSE: weighted coarse slopes / nb
    T* ph = sm + lay.phsub;

    // peers' shared memory is written before the first full cluster barrier (the pushes
    // below): arrive now, wait before the first push, so that every CTA has started
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
    __shared__ T ttp[4 * CL];                    // every rank's tip/tilt (and elongation) sums
    __shared__ T cps[CL * 2 * MAXCOARSE];        // every rank's coarse block sums (pushed)
    // the band's rows of the active-subaperture table, copied while the terms are summed
    int* msk = reinterpret_cast<int*>(sm + lay.msk);
    for (int k = threadIdx.x; k < rows * N; k += NT) cp_async(msk + k, sidx + s0 * N + k);
    // the mask and the descriptor are set-up data, read before the dependency wait; the
    // projected layers or the slopes after it
    pdl_wait();
    constexpr bool FROM_PHI = SRC == SSRC_PHI || SRC == SSRC_RESID;
    bool bad = false;                          // a non-finite measured slope (SLOPES, RESID)
    if (FROM_PHI && rows > 0) {
        // ---- V = P_g phi = sum_l (pair term of layer l) on node rows [s0, s1] ---------
        // a warp per node row; every lane's columns accumulate in the fixed layer order,
        // with the loads of several layers in flight
        constexpr int LB = (MAXNF + 1 + 31) / 32;
        const T* Vb = pb.V + static_cast<size_t>(g * d.n_layers) * pb.vslot;
        for (int ia = warp; ia < rows + 1; ia += nwarp) {
            const T* row = Vb + (s0 + ia) * pb.vs + lane;
            T acc[LB];
#pragma unroll
            for (int u = 0; u < LB; ++u) acc[u] = T(0);
            T t[MAXL][LB];
#pragma unroll
            for (int l = 0; l < MAXL; ++l)
#pragma unroll
                for (int u = 0; u < LB; ++u)
                    t[l][u] = (l < d.n_layers && lane + 32 * u < NP) ? row[static_cast<size_t>(l) * pb.vslot + 32 * u]
                                                                     : T(0);
#pragma unroll
            for (int l = 0; l < MAXL; ++l)
#pragma unroll
                for (int u = 0; u < LB; ++u)
                    if (l < d.n_layers) acc[u] += t[l][u];
#pragma unroll
            for (int u = 0; u < LB; ++u)
                if (lane + 32 * u < NP) V[ia * NP + lane + 32 * u] = acc[u];
        }
        cp_async_wait();
        __syncthreads();
        // ---- Gamma_g on the band's active subapertures -----------------------------------
        for (int ii = warp; ii < rows; ii += nwarp)
        for (int j = lane; j < N; j += 32) {
            const int k = ii * N + j;
            T sx = T(0), sy = T(0);
            const int id = msk[ii * N + j];
            if (id >= 0) {
                const T v00 = V[ii * NP + j], v01 = V[ii * NP + j + 1];
                const T v10 = V[(ii + 1) * NP + j], v11 = V[(ii + 1) * NP + j + 1];
                sx = T(0.5) * ((v01 - v00) + (v11 - v10));
                sy = T(0.5) * ((v10 - v00) + (v11 - v01));
                if (SRC == SSRC_RESID && W.nb == 1) {
                    // residual of an ordinary sensor: measured minus modelled slope (a coarse
                    // sensor's measurement enters after its block sums, below)
                    const T mx = a.in[W.soff + id], my = a.in[W.soff + W.n_active + id];
                    bad |= !(isfinite(mx) && isfinite(my));
                    sx = mx - sx;
                    sy = my - sy;
                }
            }
            SX[k] = sx;
            SY[k] = sy;
        }
    } else if (SRC == SSRC_SLOPES && rows > 0) {
        const T* s = a.in + W.soff;
        cp_async_wait();
        __syncthreads();
        for (int k = threadIdx.x; k < rows * N; k += NT) {
            const int id = msk[k];
            T sx = T(0), sy = T(0);
            if (id >= 0) {
                sx = s[id];
                sy = s[W.n_active + id];
                bad |= !(isfinite(sx) && isfinite(sy));
                if (W.nb > 1) {        // coarse: (1/nb) sigma^-2 s_K on each active fine one
                    sx *= nbinv * inv;
                    sy *= nbinv * inv;
                }
            }
            SX[k] = sx;
            SY[k] = sy;
        }
    }
    if (bad && a.status) atomicOr(a.status, 1u);
    cp_async_wait();
    __syncthreads();

    // ---- cluster reductions (fixed order): LGS tip/tilt sums, coarse block sums -------
    const bool need_tt = W.lgs;
    const bool need_coarse = FROM_PHI && W.nb > 1;
    asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");
    if (need_tt) {
        T tx = T(0), ty = T(0), ex = T(0), ey = T(0);
        for (int k = threadIdx.x; k < rows * N; k += NT) {
            tx += SX[k];
            ty += SY[k];
        }
        cta_sum2_t(tx, ty, red);
        if (W.el) {
            // spot elongation (Eq. 3): the sums of gamma beta (beta . s) as well
            for (int k = threadIdx.x; k < rows * N; k += NT) {
                if (msk[k] >= 0) {
                    const int ii = k / N;
                    T b1, b2, gam;
                    elong(W, s0 + ii, k - ii * N, b1, b2, gam);
                    const T bs = b1 * SX[k] + b2 * SY[k];
                    ex += gam * b1 * bs;
                    ey += gam * b2 * bs;
                }
            }
            cta_sum2_t(ex, ey, red);
        }
        if (threadIdx.x < CL) {           // push this rank's sums into every rank's table
            T* dst = cluster.map_shared_rank(ttp, static_cast<unsigned>(threadIdx.x));
            dst[4 * r] = tx;
            dst[4 * r + 1] = ty;
            dst[4 * r + 2] = ex;
            dst[4 * r + 3] = ey;
        }
    }
    if (need_coarse) {
        // per coarse block: the band's share of the fine-slope sums.  The warps split over
        // blocks and, within a block, over its rows (subset sw of SUB); the subsets' sums are
        // merged in subset order and pushed into every rank's table.
        constexpr int SUB = 4;
        __shared__ T csub[MAXCOARSE][SUB][2];
        const int ns = W.n_sub, nb = W.nb, nblk = ns * ns;
        for (int wk = warp; wk < nblk * SUB; wk += nwarp) {
            const int blk = wk % nblk, sw = wk / nblk;
            const int I = blk / ns, J = blk - I * ns;
            const int i0 = max(I * nb, s0), i1 = min((I + 1) * nb, s1);
            T sx = T(0), sy = T(0);
            for (int i = i0 + sw; i < i1; i += SUB)
                for (int j = J * nb + lane; j < (J + 1) * nb; j += 32) {
                    sx += SX[(i - s0) * N + j];
                    sy += SY[(i - s0) * N + j];
                }
            sx = warp_sum_t(sx);          // complete in lane 0 (shuffle-down tree)
            sy = warp_sum_t(sy);
            if (lane == 0) {
                csub[blk][sw][0] = sx;
                csub[blk][sw][1] = sy;
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nblk * CL; k += NT) {
            const int blk = k / CL, q = k - blk * CL;
            T sx = T(0), sy = T(0);
#pragma unroll
            for (int sw = 0; sw < SUB; ++sw) {
                sx += csub[blk][sw][0];
                sy += csub[blk][sw][1];
            }
            T* dst = cluster.map_shared_rank(cps, static_cast<unsigned>(q));   // push to rank q
            dst[r * 2 * MAXCOARSE + 2 * blk] = sx;
            dst[r * 2 * MAXCOARSE + 2 * blk + 1] = sy;
        }
    }
    if (need_tt || need_coarse) {
        cluster.sync();                                                   // partials ready
        if (need_tt) {
            // the CL ranks' sums, local after the barrier, added in rank order
            T tx = T(0), ty = T(0);
#pragma unroll
            for (int q = 0; q < CL; ++q) {
                tx += ttp[4 * q];
                ty += ttp[4 * q + 1];
            }
            const T mx = tx / T(W.n_active), my = ty / T(W.n_active);
            if (!W.el) {
                // C_hat^-1 = (I - T) sigma^-2 (I - T) = sigma^-2 (I - T) for an LGS
                for (int k = threadIdx.x; k < rows * N; k += NT) {
                    if (msk[k] >= 0) {
                        SX[k] = inv * (SX[k] - mx);
                        SY[k] = inv * (SY[k] - my);
                    }
                }
            } else {
                // elongated: C_hat^-1 s = sigma^-2 (u - gamma beta (beta . u) + g), u = s
                // minus its means m, g = (e - K m) / |M| the mean of gamma beta (beta . u)
                T ex = T(0), ey = T(0);
#pragma unroll
                for (int q = 0; q < CL; ++q) {
                    ex += ttp[4 * q + 2];
                    ey += ttp[4 * q + 3];
                }
                const T g1 = (ex - (el_K(W, 0, T()) * mx + el_K(W, 1, T()) * my)) / T(W.n_active);
                const T g2 = (ey - (el_K(W, 1, T()) * mx + el_K(W, 2, T()) * my)) / T(W.n_active);
                for (int k = threadIdx.x; k < rows * N; k += NT) {
                    if (msk[k] >= 0) {
                        const int ii = k / N;
                        T b1, b2, gam;
                        elong(W, s0 + ii, k - ii * N, b1, b2, gam);
                        const T ux = SX[k] - mx, uy = SY[k] - my;
                        const T bu = b1 * ux + b2 * uy;
                        SX[k] = inv * ((ux - gam * b1 * bu) + g1);
                        SY[k] = inv * ((uy - gam * b2 * bu) + g2);
                    }
                }
            }
        }
        if (need_coarse) {
            const int ns = W.n_sub;
            for (int blk = threadIdx.x; blk < ns * ns; blk += NT) {
                T sx = T(0), sy = T(0);
                for (int q = 0; q < CL; ++q) {
                    sx += cps[q * 2 * MAXCOARSE + 2 * blk];
                    sy += cps[q * 2 * MAXCOARSE + 2 * blk + 1];
                }
                // coarse slope = sum / nb; Gamma_coarse^T spreads sigma^-2 slope / nb.  The
                // residual form subtracts it from the block's measured slope.
                if (SRC == SSRC_RESID) {
                    const int K = d.cidx[W.cmask_off + blk];
                    T mx = T(0), my = T(0);
                    if (K >= 0) {
                        mx = a.in[W.soff + K];
                        my = a.in[W.soff + W.n_active + K];
                        if (!(isfinite(mx) && isfinite(my)) && a.status) atomicOr(a.status, 1u);
                    }
                    cw[2 * blk] = (mx - sx * nbinv) * inv * nbinv;
                    cw[2 * blk + 1] = (my - sy * nbinv) * inv * nbinv;
                } else {
                    cw[2 * blk] = sx * nbinv * inv * nbinv;
                    cw[2 * blk + 1] = sy * nbinv * inv * nbinv;
                }
            }
            __syncthreads();
            for (int ii = warp; ii < rows; ii += nwarp)
            for (int j = lane; j < N; j += 32) {
                const int k = ii * N + j;
                const int i = s0 + ii;
                T sx = T(0), sy = T(0);
                if (msk[ii * N + j] >= 0) {
                    const int blk = (i / W.nb) * W.n_sub + j / W.nb;
                    sx = cw[2 * blk];
                    sy = cw[2 * blk + 1];
                }
                SX[k] = sx;
                SY[k] = sy;
            }
        }
    } else if (W.nb == 1) {
        // NGS: C^-1 = sigma^-2 I
        for (int k = threadIdx.x; k < rows * N; k += NT) {
            SX[k] *= inv;
            SY[k] *= inv;
        }
    }
    cluster.sync();                                                       // weighted slopes ready
    pdl_trigger();
    // ---- Gamma_g^T on node rows [s0, s1) (and row N on the last band) --------------------
    if (rows > 0) {
        if (r > 0) {
            const T* px = cluster.map_shared_rank(SX, r - 1);
            const T* py = cluster.map_shared_rank(SY, r - 1);
            const int prow = (s0 - 1) - (r - 1) * sr;     // last row of the previous band
            for (int j = threadIdx.x; j < N; j += NT) {
                halo[j] = px[prow * N + j];
                halo[N + j] = py[prow * N + j];
            }
        } else {
            for (int j = threadIdx.x; j < N; j += NT) {
                halo[j] = T(0);
                halo[N + j] = T(0);
            }
        }
        __syncthreads();
        const int nrows = (s1 == N) ? rows + 1 : rows;
        for (int ia = warp; ia < nrows; ia += nwarp)
        for (int b = lane; b < NP; b += 32) {
            const int aa = s0 + ia;
            // subaperture row aa (below the node) and aa - 1 (above)
            const bool has0 = aa < N, c0 = b < N, c1 = b > 0;
            const T* x0 = SX + ia * N;
            const T* y0 = SY + ia * N;
            const T* x1 = ia > 0 ? SX + (ia - 1) * N : halo;
            const T* y1 = ia > 0 ? SY + (ia - 1) * N : halo + N;
            const bool has1 = aa > 0;
            const T x_ab = (has0 && c0) ? x0[b] : T(0);
            const T x_ab1 = (has0 && c1) ? x0[b - 1] : T(0);
            const T x_a1b = (has1 && c0) ? x1[b] : T(0);
            const T x_a1b1 = (has1 && c1) ? x1[b - 1] : T(0);
            const T y_ab = (has0 && c0) ? y0[b] : T(0);
            const T y_ab1 = (has0 && c1) ? y0[b - 1] : T(0);
            const T y_a1b = (has1 && c0) ? y1[b] : T(0);
            const T y_a1b1 = (has1 && c1) ? y1[b - 1] : T(0);
            a.out[W.node_off + aa * NP + b] =
                T(0.5) * ((x_ab1 - x_ab) + (x_a1b1 - x_a1b)) + T(0.5) * ((y_a1b - y_ab) + (y_a1b1 - y_ab1));
        }
    }
    cluster.sync();                                                       // neighbours done reading
}

template <class T, int SRC>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(cblk<T>(), 1)
    k_cl_sensor(__grid_constant__ const Desc<T> d, __grid_constant__ const SensorArgs<T> a,
                __grid_constant__ const SensorLayout lay, __grid_constant__ const PairBufs<T> pb) {
    cl_sensor_body<T, SRC>(d, a, lay, pb, blockIdx.y);
}

}  // namespace fewha
