// Host-side check of the CUDA path's set-up tables: build_setup and prior_diag (the C++
// code whose tables every kernel reads) run on the CPU and copied out, so that the tests can
// compare them with the oracle's matrices without a GPU.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../paper_2202_11945_gb300/csrc/fewha_internal.h"

using namespace fewha;

namespace {

template <class X>
void put(X* dst, const std::vector<X>& src) {
    if (dst && !src.empty()) std::memcpy(dst, src.data(), src.size() * sizeof(X));
}

}  // namespace

// sizes[0..7] = n_c, n_s, n_nodes, n_act, |sidx|, |cidx|, |pi0y|, |ry_lo|;
// limits[0..5] = MAXG, MAXL, MAXM, TAB, MAXN, MAXNACT (the table strides)
extern "C" int setup_sizes(const fewha_telescope* tel, const fewha_wfs* wfs, int n_wfs, const fewha_layer* layers,
                           int n_layers, const fewha_dm* dms, int n_dms, long* sizes, int* limits) {
    HostSetup s;
    std::string err;
    const int rc = build_setup(*tel, wfs, n_wfs, layers, n_layers, dms, n_dms, s, err);
    limits[0] = MAXG;
    limits[1] = MAXL;
    limits[2] = MAXM;
    limits[3] = TAB;
    limits[4] = MAXN;
    limits[5] = MAXNACT;
    if (rc) return rc;
    sizes[0] = s.n_c;
    sizes[1] = s.n_s;
    sizes[2] = s.n_nodes;
    sizes[3] = s.n_act;
    sizes[4] = static_cast<long>(s.sidx.size());
    sizes[5] = static_cast<long>(s.cidx.size());
    sizes[6] = static_cast<long>(s.pi0y.size());
    sizes[7] = static_cast<long>(s.ry_lo.size());
    return 0;
}

extern "C" int setup_tables(const fewha_telescope* tel, const fewha_wfs* wfs, int n_wfs, const fewha_layer* layers,
                            int n_layers, const fewha_dm* dms, int n_dms, double r0, double L0, int* pi0y,
                            int* pi0x, double* pfy,
                            double* pfx, int* ry_lo, int* ry_hi, int* rx_lo, int* rx_hi, int* sidx, int* cidx,
                            int* di0, double* dfw, int* dr_lo, int* dr_hi, double* fitw, double* D, double* taps) {
    HostSetup s;
    std::string err;
    const int rc = build_setup(*tel, wfs, n_wfs, layers, n_layers, dms, n_dms, s, err);
    if (rc) return rc;
    put(pi0y, s.pi0y);
    put(pi0x, s.pi0x);
    put(pfy, s.pfy);
    put(pfx, s.pfx);
    put(ry_lo, s.ry_lo);
    put(ry_hi, s.ry_hi);
    put(rx_lo, s.rx_lo);
    put(rx_hi, s.rx_hi);
    put(sidx, s.sidx);
    put(cidx, s.cidx);
    put(di0, s.di0);
    put(dfw, s.dfw);
    put(dr_lo, s.dr_lo);
    put(dr_hi, s.dr_hi);
    for (int m = 0; m < MAXM; ++m)
        for (int l = 0; l < MAXL; ++l) fitw[m * MAXL + l] = s.fitw[m][l];
    std::vector<double> d;
    prior_diag(s, s.layer_w, r0, L0, d);
    put(D, d);
    for (int k = 0; k < 6; ++k) {
        taps[k] = s.taps_h[k];
        taps[6 + k] = s.taps_g[k];
    }
    return 0;
}

// The closed loop's DM stencils of each (sensor, DM) pair, entry (g * MAXM + m) * TAB + a,
// and, after set_elongation(alpha_eta), per sensor the ten elongation constants (on flag,
// k, c, launch x and y, first midpoint, pitch, K11, K12, K22) at g * 10.
extern "C" int setup_extra(const fewha_telescope* tel, const fewha_wfs* wfs, int n_wfs, const fewha_layer* layers,
                           int n_layers, const fewha_dm* dms, int n_dms, double alpha_eta, int* qi0y, int* qi0x,
                           double* qfy, double* qfx, double* el) {
    HostSetup s;
    std::string err;
    const int rc = build_setup(*tel, wfs, n_wfs, layers, n_layers, dms, n_dms, s, err);
    if (rc) return rc;
    put(qi0y, s.qi0y);
    put(qi0x, s.qi0x);
    put(qfy, s.qfy);
    put(qfx, s.qfx);
    set_elongation(s, alpha_eta);
    for (size_t g = 0; g < s.G.size(); ++g) {
        const WfsInfo& W = s.G[g];
        const double v[10] = {double(W.el), W.el_k, W.el_c, W.el_lx, W.el_ly, W.el_x0, W.el_d,
                              W.el_K11, W.el_K12, W.el_K22};
        for (int q = 0; q < 10; ++q) el[g * 10 + q] = v[q];
    }
    return 0;
}

// The 8 x 8 tail matrix of the wavelet kernels (row stride 64 here); 0 if its synthesis
// check failed.
extern "C" int setup_tail(double* A) {
    double h[6], g[6];
    db3_taps(h, g);
    const std::vector<double> t = tail_operator(h, g, 64);
    if (t.empty()) return -1;
    put(A, t);
    return 0;
}

// The 1-D wavelet basis tables of the exact Jacobi diagonal: basis (all functions
// concatenated) and basis_off (MAXL * (MAXLEV + 1) * 2 offsets, basis_index(l, j, kind)).
extern "C" int setup_basis(const fewha_telescope* tel, const fewha_wfs* wfs, int n_wfs, const fewha_layer* layers,
                           int n_layers, const fewha_dm* dms, int n_dms, double* basis, long n_basis,
                           int* basis_off, int* maxlev) {
    HostSetup s;
    std::string err;
    const int rc = build_setup(*tel, wfs, n_wfs, layers, n_layers, dms, n_dms, s, err);
    if (rc) return rc;
    *maxlev = MAXLEV;
    if (static_cast<long>(s.basis.size()) != n_basis) return -100;
    put(basis, s.basis);
    put(basis_off, s.basis_off);
    return 0;
}
