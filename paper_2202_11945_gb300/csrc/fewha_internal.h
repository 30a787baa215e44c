// Internal descriptors shared by the host set-up code and the CUDA kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fewha.h"

namespace fewha {

constexpr int MAXL = FEWHA_MAX_LAYERS;
constexpr int MAXG = FEWHA_MAX_WFS;
constexpr int MAXM = FEWHA_MAX_DMS;
constexpr int MAXN = FEWHA_MAX_GRID;
constexpr int MAXNF = FEWHA_MAX_NFINE;
constexpr int MAXNACT = 2 * MAXN;       // actuators per DM side
constexpr int TAB = MAXNF + 1;          // projection table stride per (sensor, layer)
constexpr int MAXCOARSE = FEWHA_MAX_COARSE * FEWHA_MAX_COARSE;

struct LayerInfo {
    int n;        // grid side (power of two)
    int log2n;
    int levels;   // wavelet levels
    int off;      // offset in coefficient / layer vectors
    int full;     // levels == log2n: the LL band is the single piston coefficient
};

struct WfsInfo {
    int N;          // fine subapertures per side (n_sub * nb)
    int nb;         // fine per coarse (1: ordinary sensor)
    int n_sub;      // subapertures per side as measured
    int lgs;        // tip/tilt removed (Sec. 3.2)
    int n_active;   // active measured subapertures
    int soff;       // offset of its slopes
    int node_off;   // offset of its (N+1)^2 aperture nodes
    int mask_off;   // offset of its N*N slope-index table
    int cmask_off;  // offset of its n_sub^2 coarse-index table (nb > 1)
    double sig2inv; // 1 / sigma^2
    // LGS spot elongation (Eq. 3): subaperture (i, j) has beta = el_k ((el_x0 + j el_d,
    // el_x0 + i el_d) - (el_lx, el_ly)) and C_ij^-1 = sigma^-2 (I - gamma beta beta^T),
    // gamma = el_c / (1 + el_c |beta|^2); el_K = sum of gamma beta beta^T over the
    // active subapertures
    int el;
    double el_k, el_c, el_lx, el_ly, el_x0, el_d;
    double el_K11, el_K12, el_K22;
    // the same nine constants in single precision (k, c, lx, ly, x0, d, K11, K12, K22), so
    // that the FP32 kernels convert nothing (GB300's FP64 pipe, conversions included,
    // runs at ~1/64 of the FP32 rate)
    float el_f[9];
};

struct DmInfo {
    int n_act;
    int off;
};

// Everything a kernel needs about one instance, passed by value.
template <class T>
struct alignas(16) Desc {   // 16-byte multiple: batched kernels copy it in 16-byte chunks
    int n_layers, n_wfs, n_dms;
    int n_c, n_s, n_nodes, n_act;
    int max_n, max_N;
    LayerInfo L[MAXL];
    WfsInfo G[MAXG];
    DmInfo Mi[MAXM];
    T fitw[MAXM][MAXL];   // share of layer l given to DM m
    T alpha, gain;
    // P_g tables, pair (g, l) at (g * MAXL + l) * TAB: grid row/col of node a and weight
    const int* pi0y;
    const int* pi0x;
    const T* pfy;
    const T* pfx;
    // P_g^T gather ranges, pair (g, l) at (g * MAXL + l) * MAXN: aperture rows/cols
    // touching layer row/col i are [lo, hi)
    const int* ry_lo;
    const int* ry_hi;
    const int* rx_lo;
    const int* rx_hi;
    // slope index tables (see WfsInfo)
    const int* sidx;
    const int* cidx;
    // DM fit tables, pair (m, l) at (m * MAXL + l) * MAXNACT
    const int* di0;
    const T* dfw;
    // F^T gather ranges, pair (m, l) at (m * MAXL + l) * MAXN
    const int* dr_lo;
    const int* dr_hi;
    // per-coefficient diagonals
    const T* D;
    const T* Jinv;
    // D per (layer, level): detail level k = 1 .. levels (1 the finest), levels + 1 the LL band
    T Dlev[MAXL][9];
    const T* tailop;   // analysis of the 8 x 8 tail levels (64 x TAIL_LD), or null
    // footprint box of each (sensor, layer) pair: row0, rows, col0, cols (16-byte aligned
    // column superset); kept in the descriptor so that warps read it from the constant bank
    int box[MAXG][MAXL][4];
};

// Host-side result of geometry set-up (all in double).
struct HostSetup {
    std::vector<LayerInfo> L;
    std::vector<WfsInfo> G;
    std::vector<DmInfo> Mi;
    std::vector<double> layer_h, layer_w, layer_delta;
    std::vector<double> dlev;           // D per (layer, level), MAXL * (MAXLEV + 1) (see Desc::Dlev)
    std::vector<double> wfs_sigma;
    double fitw[MAXM][MAXL];
    int n_c = 0, n_s = 0, n_nodes = 0, n_act = 0, max_n = 0, max_N = 0;
    std::vector<int> pi0y, pi0x;        // MAXG*MAXL*TAB
    std::vector<double> pfy, pfx;
    std::vector<int> ry_lo, ry_hi, rx_lo, rx_hi;   // MAXG*MAXL*MAXN
    std::vector<int> sidx, cidx;
    std::vector<int> di0;               // MAXM*MAXL*MAXNACT
    std::vector<double> dfw;
    std::vector<int> dr_lo, dr_hi;      // MAXM*MAXL*MAXN
    // DM m seen by sensor g (closed loop), pair (g, m) at (g * MAXM + m) * TAB: actuator
    // row/col index of node a (the stencil {i0, i0 + 1} may leave the lattice) and weight
    std::vector<int> qi0y, qi0x;
    std::vector<double> qfy, qfx;
    bool dm_proj_ok = true;             // every DM below every LGS
    // per sensor: launch position, sodium FWHM, spot FWHM, LGS height (spot elongation)
    std::vector<double> wfs_lx, wfs_ly, wfs_na_fwhm, wfs_spot_fwhm, wfs_H;
    double D = 0.0;
    // 1-D wavelet basis functions at shift 0: layer l, level j (1..levels), kind 0/1
    std::vector<double> basis;
    std::vector<int> basis_off;         // MAXL * (MAXN_LEVELS + 1) * 2
    double taps_h[6], taps_g[6];
};

constexpr int MAXLEV = 8;   // log2(MAXN) + 1
static_assert(MAXLEV + 1 == 9, "Desc::Dlev holds levels 0 .. MAXLEV");
#ifdef __CUDACC__
__host__ __device__
#endif
inline int basis_index(int l, int j, int kind) { return (l * (MAXLEV + 1) + j) * 2 + kind; }

// Least-squares DM fitting over fitting directions (fewha_fit_ls), host tables in double.
// Pupil node (i, j), i, j = 0 .. n_fit, sits at (x_j, x_i), x_i = -D/2 + i D / n_fit.
struct LsfitHost {
    int n_dirs = 0;
    int nf1 = 0;                        // pupil nodes per side, n_fit + 1
    int n_pup = 0;                      // pupil nodes inside the annulus
    std::vector<unsigned char> mask;    // nf1 * nf1, row-major
    // layer l along direction k, entry (k * MAXL + l) * nf1 + i: grid row (y) / column (x)
    // i0 of the first node of the linear stencil of pupil row / column i and the weight f of
    // node i0 + 1 (node i0 has 1 - f)
    std::vector<int> ly0, lx0;
    std::vector<double> lfy, lfx;
    // DM m along direction k, entry (k * MAXM + m) * nf1 + i: the same for the actuator
    // lattice; i0 and i0 + 1 may leave it (a hat beyond the outer actuators is zero)
    std::vector<int> my0, mx0;
    std::vector<double> mfy, mfx;
    // pupil rows / columns whose stencil touches actuator row / column p of DM m along
    // direction k, entry (k * MAXM + m) * MAXNACT + p: the range [lo, hi)
    std::vector<int> ylo, yhi, xlo, xhi;
};

// Host set-up (fewha_setup.cpp).  Return FEWHA_OK or an error code with a message.
int build_setup(const fewha_telescope& tel, const fewha_wfs* wfs, int n_wfs,
                const fewha_layer* layers, int n_layers, const fewha_dm* dms, int n_dms,
                HostSetup& out, std::string& err);
void db3_taps(double h[6], double g[6]);
// Spot-elongation constants of every LGS for alpha_eta (Eq. 3); 0 turns them off.
void set_elongation(HostSetup& s, double alpha_eta);
// Tables of the least-squares fit over fitting directions (Sec. 4.1) for an instance set
// up as `s` with central obstruction ratio `obs` and DMs `dms`.  FEWHA_ERR_GEOMETRY if a
// pupil node along a direction samples a layer outside its grid.
int build_lsfit(const HostSetup& s, double obs, const fewha_dm* dms, const fewha_lsfit& cfg,
                LsfitHost& out, std::string& err);
// One periodic db3 level step on m values of stride st, analysis or synthesis (inv).
void db3_step_host(double* x, int m, int st, const double* h, const double* g, bool inv);
// The last three levels of a full decomposition (an 8 x 8 LL block down to 1 x 1) as one
// 64 x 64 analysis matrix A, entry (k, o) at k * ld + o (input k = 8 i + j to output o),
// from unit inputs through the level steps; empty unless the synthesis of the same steps is
// A^T (which the inverse kernels apply).
std::vector<double> tail_operator(const double* h, const double* g, int ld);
// Prior D (Sec. 3.1), one value per coefficient.
void prior_diag(const HostSetup& s, const std::vector<double>& weights, double r0, double L0,
                std::vector<double>& D);

}  // namespace fewha
