// Per (sensor, layer) pair kernels: the bilinear projection P_g (Sec. 2) is a sum over
// layers of separable interpolations, P_g phi = sum_l R_y,gl phi_l R_x,gl^T, and its
// adjoint is sum_g R_y,gl^T u_g R_x,gl.  One CTA per pair computes its term with two
// separable passes in shared memory; the sensor and layer kernels add the terms up.
// No reduction crosses CTAs here, so the sums stay in a fixed order.
#pragma once

#include "fewha_cluster.cuh"

namespace fewha {

// V_gl(a, b) = sum_{i,j} wy(a, i) wx(b, j) phi_l(i, j) over the pair's footprint box; NT
// threads per CTA (at least the node row length N + 1).
template <class T, int NT = cblk<T>()>
__device__ __forceinline__ void proj_body(const Desc<T>& d, const T* __restrict__ phi,
                                          const PairBufs<T>& pb, const int g, const int l) {
    constexpr int V = vec16<T>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* F = reinterpret_cast<T*>(smem_raw);       // footprint of phi_l: rows x cols
    const int N = d.G[g].N, NP = N + 1;
    const int tp = (g * MAXL + l) * TAB;
    const int r0 = d.box[g][l][0], rows = d.box[g][l][1], c0 = d.box[g][l][2], cols = d.box[g][l][3];
    const int n = d.L[l].n;
    T* Tm = F + rows * cols;                      // pass X result: rows x NP
    T* tfx = Tm + rows * NP;                      // the pair's interpolation tables (NP each)
    T* tfy = tfx + NP;
    int* tj0 = reinterpret_cast<int*>(tfy + NP);
    int* ti0 = tj0 + NP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = NT >> 5;
    // the tables travel with the footprint (async copies, all in flight together), so
    // that no pass waits on a table load from global memory
    for (int k = threadIdx.x; k < NP; k += NT) {
        cp_async(tfx + k, d.pfx + tp + k);
        cp_async(tfy + k, d.pfy + tp + k);
        cp_async(tj0 + k, d.pi0x + tp + k);
        cp_async(ti0 + k, d.pi0y + tp + k);
    }
    // the tables are set-up data, copied before the dependency wait; phi after it
    pdl_wait();
    pdl_trigger();
    const T* src = phi + d.L[l].off + r0 * n + c0;
    if ((n & (V - 1)) == 0) {
        const int cpr = cols / V;
        for (int i = warp; i < rows; i += nwarp)
            for (int c = lane; c < cpr; c += 32) cp_async16(F + i * cols + c * V, src + i * n + c * V);
    } else {
        for (int i = warp; i < rows; i += nwarp)
            for (int j = lane; j < cols; j += 32) cp_async(F + i * cols + j, src + i * n + j);
    }
    cp_async_wait();
    __syncthreads();
    // pass X: Tm(i, b) = (1 - fx_b) F(i, j0_b) + fx_b F(i, j0_b + 1); thread per column b
    {
        const int b = threadIdx.x % NP, rg = threadIdx.x / NP, groups = NT / NP;
        if (rg < groups) {
            const int j0 = tj0[b] - c0;
            const T fx = tfx[b];
            for (int i = rg; i < rows; i += groups)
                Tm[i * NP + b] = (T(1) - fx) * F[i * cols + j0] + fx * F[i * cols + j0 + 1];
        }
    }
    __syncthreads();
    // pass Y: V(a, b) = (1 - fy_a) Tm(i0_a, b) + fy_a Tm(i0_a + 1, b)
    T* out = pb.V + static_cast<size_t>(g * d.n_layers + l) * pb.vslot;
    for (int a = warp; a < NP; a += nwarp) {
        const int i0 = ti0[a] - r0;
        const T fy = tfy[a];
        for (int b = lane; b < NP; b += 32)
            out[a * pb.vs + b] = (T(1) - fy) * Tm[i0 * NP + b] + fy * Tm[(i0 + 1) * NP + b];
    }
}

template <class T>
__global__ void __launch_bounds__(cblk<T>(), 1) k_proj(__grid_constant__ const Desc<T> d,
                                                       const T* __restrict__ phi,
                                                       __grid_constant__ const PairBufs<T> pb) {
    proj_body<T>(d, phi, pb, blockIdx.x, blockIdx.y);
}

// Y_gl(i, j) = sum_{a,b} wy(a, i) wx(b, j) u_g(a, b) on the pair's footprint box.  KM >= the
// largest number of aperture rows (columns) touching one layer row (column): the loops over
// a row's taps are unrolled to KM (the weight tables keep the stride KMAX).  NT threads per
// CTA (at least the box width).
template <class T, int KM = KMAX, int NT = cblk<T>()>
__device__ __forceinline__ void projT_body(const Desc<T>& d, const T* __restrict__ u,
                                           const PairBufs<T>& pb, const int g, const int l) {
    constexpr int V = vec16<T>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* U = reinterpret_cast<T*>(smem_raw);       // u_g, (N+1)^2 (+ alignment shift)
    const int N = d.G[g].N, NP = N + 1;
    const int r0 = d.box[g][l][0], rows = d.box[g][l][1], cols = d.box[g][l][3];
    const int start = d.G[g].node_off, s0a = start & ~(V - 1);
    const int ushift = start - s0a;
    const int pr = g * d.n_layers + l;
    auto up16 = [](int x) { return (x + V - 1) & ~(V - 1); };
    T* Tx = U + up16(ushift + NP * NP);           // pass X result: NP x cols
    T* cw = Tx + up16(NP * cols);                // column weights: cols x KMAX
    T* rw = cw + cols * KMAX;                     // row weights: rows x KMAX
    int2* cinf = reinterpret_cast<int2*>(rw + rows * KMAX);   // first aperture column, count
    int2* rinf = cinf + ((cols + 1) & ~1);        // 16-byte aligned
    constexpr int I2 = sizeof(int2) / sizeof(T);  // T elements per int2
    // the pair's weight tables and u_g, 16-byte copies all in flight together; the tables
    // (set-up data) before the dependency wait, u_g after it
    stage16(cw, pb.tw + static_cast<size_t>(pr * 2) * MAXN * KMAX, cols * KMAX, threadIdx.x, NT);
    stage16(rw, pb.tw + static_cast<size_t>(pr * 2 + 1) * MAXN * KMAX, rows * KMAX, threadIdx.x, NT);
    stage16(reinterpret_cast<T*>(cinf), reinterpret_cast<const T*>(pb.ti + static_cast<size_t>(pr * 2) * MAXN),
            cols * I2, threadIdx.x, NT);
    stage16(reinterpret_cast<T*>(rinf), reinterpret_cast<const T*>(pb.ti + static_cast<size_t>(pr * 2 + 1) * MAXN),
            rows * I2, threadIdx.x, NT);
    pdl_wait();
    pdl_trigger();
    stage16(U, u + s0a, ushift + NP * NP, threadIdx.x, NT);
    cp_async_wait();
    __syncthreads();
    const T* Us = U + ushift;
    // pass X: Tx(a, j) = sum_{b touching j} wx(b, j) u(a, b); thread per box column j
    {
        const int groups = NT / cols;
        const int jj = threadIdx.x % cols, rg = threadIdx.x / cols;
        if (rg < groups) {
            const int2 ci = cinf[jj];
            T w[KM];
#pragma unroll
            for (int q = 0; q < KM; ++q) w[q] = cw[jj * KMAX + q];
            for (int a = rg; a < NP; a += groups) {
                const T* urow = Us + a * NP + ci.x;
                T acc = T(0);
#pragma unroll
                for (int q = 0; q < KM; ++q)
                    if (q < ci.y) acc += w[q] * urow[q];
                Tx[a * cols + jj] = acc;
            }
        }
    }
    __syncthreads();
    // pass Y: Y(i, j) = sum_{a touching i} wy(a, i) Tx(a, j); warp per box row i
    T* out = pb.Y + static_cast<size_t>(g * d.n_layers + l) * pb.yslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = NT >> 5;
    (void)r0;
    for (int ii = warp; ii < rows; ii += nwarp) {
        const int2 ri = rinf[ii];
        T wv[KM];
#pragma unroll
        for (int q = 0; q < KM; ++q) wv[q] = rw[ii * KMAX + q];
        for (int jj = lane; jj < cols; jj += 32) {
            const T* tcol = Tx + ri.x * cols + jj;
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < KM; ++q)
                if (q < ri.y) acc += wv[q] * tcol[q * cols];
            out[ii * cols + jj] = acc;
        }
    }
}

template <class T, int KM>
__global__ void __launch_bounds__(cblk<T>(), 1) k_projT(__grid_constant__ const Desc<T> d,
                                                        const T* __restrict__ u,
                                                        __grid_constant__ const PairBufs<T> pb) {
    projT_body<T, KM>(d, u, pb, blockIdx.x, blockIdx.y);
}

}  // namespace fewha
