// Least-squares DM fitting over fitting directions (Sec. 4.1: with more reconstructed
// layers than DMs the fitting step becomes a least-squares problem of its own).
//
// The commands a minimise sum_k w_k ||Pi (A_k a - L_k phi)||^2 + eps ||a||^2: along
// fitting direction k the pupil nodes see the layers phi (L_k, linear stencils on the
// layer grids) and the DMs (A_k, bilinear actuator hats), and Pi removes the mean over
// the pupil nodes.  The normal equations N a = sum_k w_k A_k^T Pi L_k phi,
// N = sum_k w_k A_k^T Pi A_k + eps I, are solved by CG.  One CG step is three kernels:
//   k_lsf_sample<DM>  a grid of (slices, directions): u_k = A_k p on the pupil nodes of a
//                     slice (zero off the pupil) and the slice's sum of u_k in double;
//   k_lsf_adj         one thread per actuator: the means of the u_k from the slice sums in
//                     a fixed order, then q = sum_k w_k A_k^T Pi u_k + eps p, gathered over
//                     the pupil rows and columns whose stencils touch the actuator
//                     (host-built ranges, no atomics; Pi applied on the fly), and per-CTA
//                     shares of p.q;
//   k_lsf_cg          one CTA: the p.q total in a fixed order, the CG step, r.r.
// The right-hand side is k_lsf_sample<LAYER> on phi followed by k_lsf_adj without p.
// Once the CG has stopped (state[0] != 0) the kernels of the remaining steps of a chunk
// return at once.
#pragma once

#include "fewha_internal.h"

namespace fewha {

constexpr int LSF_SBLK = 256;    // k_lsf_sample: threads per slice of a direction's pupil grid
constexpr int LSF_MAXSL = 304;   // most (direction, slice) CTAs of k_lsf_sample (2 per SM)
constexpr int LSF_ABLK = 256;    // k_lsf_adj: actuators per CTA
constexpr int LSF_CBLK = 1024;   // k_lsf_cg: the single CTA
constexpr int LSF_MAXK = FEWHA_MAX_FIT_DIRS;

template <class T>
struct LsDesc {
    int n_dirs, nf1, n_pup, n_layers, n_dms, n_a;
    int n_slices;                        // k_lsf_sample CTAs per direction
    int lay_n[MAXL], lay_off[MAXL];
    int dm_n[MAXM], dm_off[MAXM];
    T w[LSF_MAXK];
    T eps;
    const unsigned char* mask;           // nf1 * nf1 pupil nodes
    const int *ly0, *lx0, *my0, *mx0;    // see LsfitHost
    const T *lfy, *lfx, *mfy, *mfx;
    const int *ylo, *yhi, *xlo, *xhi;
};

// Value at pupil node (i, j) along direction k of the layers (LAYER) or the DMs: the sum
// over the sources of the separable two-point stencils.  Taps outside a DM lattice are
// zero; layer stencils never leave their grid (checked at set-up).
template <class T, bool LAYER>
__host__ __device__ inline T lsf_sample(const LsDesc<T>& d, const T* src, int k, int i, int j) {
    T val = T(0);
    const int ns = LAYER ? d.n_layers : d.n_dms;
    for (int s = 0; s < ns; ++s) {
        const int n = LAYER ? d.lay_n[s] : d.dm_n[s];
        const T* g = src + (LAYER ? d.lay_off[s] : d.dm_off[s]);
        const int e = (k * (LAYER ? MAXL : MAXM) + s) * d.nf1;
        const int y0 = (LAYER ? d.ly0 : d.my0)[e + i];
        const int x0 = (LAYER ? d.lx0 : d.mx0)[e + j];
        const T fy = (LAYER ? d.lfy : d.mfy)[e + i];
        const T fx = (LAYER ? d.lfx : d.mfx)[e + j];
        const T wy[2] = {T(1) - fy, fy};
        const T wx[2] = {T(1) - fx, fx};
        for (int t = 0; t < 2; ++t) {
            const int r = y0 + t;
            if (r < 0 || r >= n) continue;
            T row = T(0);
            for (int u = 0; u < 2; ++u) {
                const int c = x0 + u;
                if (c < 0 || c >= n) continue;
                row += wx[u] * g[r * n + c];
            }
            val += wy[t] * row;
        }
    }
    return val;
}

// (sum_k w_k A_k^T Pi u_k) at actuator (p, q) of DM m, u_k zero off the pupil and mean[k]
// its mean over the pupil nodes: the pupil rows [ylo, yhi) and columns [xlo, xhi) are those
// whose stencils include the actuator; its hat weight in each is the stencil weight on that
// actuator.
template <class T>
__host__ __device__ inline T lsf_adjoint(const LsDesc<T>& d, const T* v, const T* mean, int m, int p, int q) {
    T acc = T(0);
    const int nf1 = d.nf1;
    for (int k = 0; k < d.n_dirs; ++k) {
        const int e = k * MAXM + m;
        const int ylo = d.ylo[e * MAXNACT + p], yhi = d.yhi[e * MAXNACT + p];
        const int xlo = d.xlo[e * MAXNACT + q], xhi = d.xhi[e * MAXNACT + q];
        const T* vk = v + static_cast<size_t>(k) * nf1 * nf1;
        const T mk = mean[k];
        T sk = T(0);
        for (int i = ylo; i < yhi; ++i) {
            const int y0 = d.my0[e * nf1 + i];
            const T fy = d.mfy[e * nf1 + i];
            const T wy = y0 == p ? T(1) - fy : fy;   // y0 is p or p - 1 inside the range
            T row = T(0);
            for (int j = xlo; j < xhi; ++j) {
                const int x0 = d.mx0[e * nf1 + j];
                const T fx = d.mfx[e * nf1 + j];
                const int g = i * nf1 + j;
                row += (x0 == q ? T(1) - fx : fx) * (vk[g] - mk * static_cast<T>(d.mask[g]));
            }
            sk += wy * row;
        }
        acc += d.w[k] * sk;
    }
    return acc;
}

#ifdef __CUDACC__

// Sum over the CTA in a fixed order; every thread gets the total.  All threads call it.
template <int BLK>
__device__ __forceinline__ double lsf_block_sum(double v) {
    __shared__ double sh[BLK / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();                 // sh may still be read from an earlier call
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < BLK / 32; ++w) t += sh[w];
    return t;
}

// u_k = A_k src (DMs) or L_k src (layers) on slice blockIdx.x of the nf1 x nf1 pupil grid
// of direction k = blockIdx.y, zero off the pupil, and the slice's sum of u_k (msum).
template <class T, bool LAYER>
__global__ void __launch_bounds__(LSF_SBLK) k_lsf_sample(LsDesc<T> d, const T* src, T* v, double* msum,
                                                         const int* state) {
    if (state && state[0]) return;
    const int k = blockIdx.y;
    const int nf1 = d.nf1, npix = nf1 * nf1;
    const int chunk = (npix + d.n_slices - 1) / d.n_slices;
    const int g0 = blockIdx.x * chunk, g1 = min(npix, g0 + chunk);
    T* vk = v + static_cast<size_t>(k) * npix;
    double acc = 0.0;
    for (int g = g0 + threadIdx.x; g < g1; g += LSF_SBLK) {
        T val = T(0);
        if (d.mask[g]) {
            const int i = g / nf1;
            val = lsf_sample<T, LAYER>(d, src, k, i, g - i * nf1);
            acc += static_cast<double>(val);
        }
        vk[g] = val;
    }
    const double t = lsf_block_sum<LSF_SBLK>(acc);
    if (threadIdx.x == 0) msum[k * d.n_slices + blockIdx.x] = t;
}

// out = sum_k w_k A_k^T Pi u_k (+ eps x, and the CTA's share of x.out into part, when x is
// given); the mean of u_k is its slice sums (msum) added in slice order over n_pup.
template <class T>
__global__ void __launch_bounds__(LSF_ABLK) k_lsf_adj(LsDesc<T> d, const T* v, const double* msum, const T* x,
                                                      T* out, double* part, const int* state) {
    if (state && state[0]) return;
    __shared__ T s_mean[LSF_MAXK];
    if (threadIdx.x < d.n_dirs) {
        double t = 0.0;
        for (int sl = 0; sl < d.n_slices; ++sl) t += msum[threadIdx.x * d.n_slices + sl];
        s_mean[threadIdx.x] = static_cast<T>(t / d.n_pup);
    }
    __syncthreads();
    const int a = blockIdx.x * LSF_ABLK + threadIdx.x;
    double pq = 0.0;
    if (a < d.n_a) {
        int m = 0;
        while (m + 1 < d.n_dms && a >= d.dm_off[m + 1]) ++m;
        const int n = d.dm_n[m], loc = a - d.dm_off[m];
        const int p = loc / n;
        T val = lsf_adjoint<T>(d, v, s_mean, m, p, loc - p * n);
        if (x) {
            const T xa = x[a];
            val += d.eps * xa;
            pq = static_cast<double>(xa) * static_cast<double>(val);
        }
        out[a] = val;
    }
    if (part) {
        const double t = lsf_block_sum<LSF_ABLK>(pq);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

template <class T>
struct LsCg {
    int n, nparts, max_iters;
    double tol2;          // stop once r.r <= tol2 * (r.r at the start)
    T *a, *r, *p;
    const T* q;           // N p (a step) or the right-hand side (the start)
    const double* part;   // per-CTA shares of p.q
    double* sc;           // [0] r.r, [1] r.r at the start
    int* state;           // [0] 0 running, 1 stopped, 2 p.q <= 0 or not a number; [1] steps run
};

// START: a = 0, r = p = b, r.r.  Otherwise one CG step on N (double scalars).
template <class T, bool START>
__global__ void __launch_bounds__(LSF_CBLK) k_lsf_cg(LsCg<T> g) {
    __shared__ double s_pq;
    const int t = threadIdx.x;
    if (START) {
        double rr = 0.0;
        for (int i = t; i < g.n; i += LSF_CBLK) {
            const T b = g.q[i];
            g.a[i] = T(0);
            g.r[i] = b;
            g.p[i] = b;
            rr += static_cast<double>(b) * static_cast<double>(b);
        }
        rr = lsf_block_sum<LSF_CBLK>(rr);
        if (t == 0) {
            g.sc[0] = rr;
            g.sc[1] = rr;
            g.state[0] = (rr == 0.0 || g.max_iters <= 0) ? 1 : 0;
            g.state[1] = 0;
        }
        return;
    }
    if (g.state[0]) return;
    if (t == 0) {
        double pq = 0.0;
        for (int j = 0; j < g.nparts; ++j) pq += g.part[j];
        s_pq = pq;
    }
    __syncthreads();
    const double pq = s_pq, rr = g.sc[0];
    if (!(pq > 0.0)) {
        if (t == 0) g.state[0] = 2;
        return;
    }
    const T al = static_cast<T>(rr / pq);
    double rn = 0.0;
    for (int i = t; i < g.n; i += LSF_CBLK) {
        const T ri = g.r[i] - al * g.q[i];
        g.a[i] += al * g.p[i];
        g.r[i] = ri;
        rn += static_cast<double>(ri) * static_cast<double>(ri);
    }
    rn = lsf_block_sum<LSF_CBLK>(rn);
    const T beta = static_cast<T>(rn / rr);
    for (int i = t; i < g.n; i += LSF_CBLK) g.p[i] = g.r[i] + beta * g.p[i];
    if (t == 0) {
        const int it = g.state[1] + 1;
        g.state[1] = it;
        g.sc[0] = rn;
        if (!(rn > g.tol2 * g.sc[1]) || it >= g.max_iters) g.state[0] = 1;
    }
}

#endif  // __CUDACC__

}  // namespace fewha
