// Host-side check of the least-squares fit's CUDA path: the tables of build_lsfit and the
// per-element functions of fewha_lsfit.cuh (the ones the kernels call per pupil node and
// per actuator) evaluated on the CPU, slice by slice and actuator by actuator as the
// kernels do, so that the index arithmetic can be compared with the oracle without a GPU.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../paper_2202_11945_gb300/csrc/fewha_lsfit.cuh"

using namespace fewha;

namespace {

struct Ctx {
    HostSetup S;
    LsfitHost L;
    LsDesc<double> d{};
    std::vector<double> msum;
};

int setup(Ctx& c, const fewha_telescope* tel, const fewha_wfs* wfs, int n_wfs, const fewha_layer* layers,
          int n_layers, const fewha_dm* dms, int n_dms, const fewha_lsfit* cfg) {
    std::string err;
    int rc = build_setup(*tel, wfs, n_wfs, layers, n_layers, dms, n_dms, c.S, err);
    if (rc) return rc;
    if ((rc = build_lsfit(c.S, tel->obs, dms, *cfg, c.L, err))) return rc;
    LsDesc<double>& d = c.d;
    d.n_dirs = c.L.n_dirs;
    d.nf1 = c.L.nf1;
    d.n_pup = c.L.n_pup;
    d.n_layers = n_layers;
    d.n_dms = n_dms;
    d.n_a = c.S.n_act;
    d.n_slices = std::max(1, std::min((d.nf1 * d.nf1 + LSF_SBLK - 1) / LSF_SBLK, LSF_MAXSL / d.n_dirs));
    for (int l = 0; l < n_layers; ++l) {
        d.lay_n[l] = c.S.L[l].n;
        d.lay_off[l] = c.S.L[l].off;
    }
    for (int m = 0; m < n_dms; ++m) {
        d.dm_n[m] = c.S.Mi[m].n_act;
        d.dm_off[m] = c.S.Mi[m].off;
    }
    for (int k = 0; k < d.n_dirs; ++k) d.w[k] = cfg->weight[k];
    d.eps = cfg->eps;
    d.mask = c.L.mask.data();
    d.ly0 = c.L.ly0.data();
    d.lx0 = c.L.lx0.data();
    d.my0 = c.L.my0.data();
    d.mx0 = c.L.mx0.data();
    d.lfy = c.L.lfy.data();
    d.lfx = c.L.lfx.data();
    d.mfy = c.L.mfy.data();
    d.mfx = c.L.mfx.data();
    d.ylo = c.L.ylo.data();
    d.yhi = c.L.yhi.data();
    d.xlo = c.L.xlo.data();
    d.xhi = c.L.xhi.data();
    c.msum.assign(static_cast<size_t>(d.n_dirs) * d.n_slices, 0.0);
    return 0;
}

// k_lsf_sample: u_k on every slice, zero off the pupil, and the slice sums
template <bool LAYER>
void sample(Ctx& c, const double* src, double* v) {
    const LsDesc<double>& d = c.d;
    const int npix = d.nf1 * d.nf1, chunk = (npix + d.n_slices - 1) / d.n_slices;
    for (int k = 0; k < d.n_dirs; ++k)
        for (int sl = 0; sl < d.n_slices; ++sl) {
            double acc = 0.0;
            for (int g = sl * chunk; g < std::min(npix, (sl + 1) * chunk); ++g) {
                double val = 0.0;
                if (d.mask[g]) {
                    const int i = g / d.nf1;
                    val = lsf_sample<double, LAYER>(d, src, k, i, g - i * d.nf1);
                    acc += val;
                }
                v[static_cast<size_t>(k) * npix + g] = val;
            }
            c.msum[k * d.n_slices + sl] = acc;
        }
}

// k_lsf_adj: the pupil means from the slice sums, then the gathered adjoint (+ eps x)
void adjoint(Ctx& c, const double* v, const double* x, double* out) {
    const LsDesc<double>& d = c.d;
    double mean[LSF_MAXK];
    for (int k = 0; k < d.n_dirs; ++k) {
        double t = 0.0;
        for (int sl = 0; sl < d.n_slices; ++sl) t += c.msum[k * d.n_slices + sl];
        mean[k] = t / d.n_pup;
    }
    for (int a = 0; a < d.n_a; ++a) {
        int m = 0;
        while (m + 1 < d.n_dms && a >= d.dm_off[m + 1]) ++m;
        const int n = d.dm_n[m], loc = a - d.dm_off[m], p = loc / n;
        double val = lsf_adjoint<double>(d, v, mean, m, p, loc - p * n);
        if (x) val += d.eps * x[a];
        out[a] = val;
    }
}

}  // namespace

// u_layers = L_k phi, u_dms = A_k a on the pupil grids (not centred; zero off the pupil),
// their pupil means (K each), and out = sum_k w_k A_k^T Pi A_k a + eps a.
extern "C" int lsfit_host_apply(const fewha_telescope* tel, const fewha_wfs* wfs, int n_wfs,
                                const fewha_layer* layers, int n_layers, const fewha_dm* dms, int n_dms,
                                const fewha_lsfit* cfg, const double* phi, const double* a, double* u_layers,
                                double* mean_layers, double* u_dms, double* mean_dms, double* out) {
    Ctx c;
    int rc = setup(c, tel, wfs, n_wfs, layers, n_layers, dms, n_dms, cfg);
    if (rc) return rc;
    const int K = c.d.n_dirs, S = c.d.n_slices;
    auto means = [&](double* m) {
        for (int k = 0; k < K; ++k) {
            double t = 0.0;
            for (int sl = 0; sl < S; ++sl) t += c.msum[k * S + sl];
            m[k] = t / c.d.n_pup;
        }
    };
    sample<true>(c, phi, u_layers);
    means(mean_layers);
    sample<false>(c, a, u_dms);
    means(mean_dms);
    adjoint(c, u_dms, a, out);
    return 0;
}

namespace {

// The CG of fewha_fit_ls step by step (k_lsf_cg's arithmetic: vectors and operators in T,
// inner products and scalars in double), with the operators evaluated as above.
template <class T>
int solve(const fewha_telescope* tel, const fewha_wfs* wfs, int n_wfs, const fewha_layer* layers, int n_layers,
          const fewha_dm* dms, int n_dms, const fewha_lsfit* cfg, const double* phi64, double* a64, double tol,
          int max_iters, int* iters, double* rel) {
    Ctx c;
    int rc = setup(c, tel, wfs, n_wfs, layers, n_layers, dms, n_dms, cfg);
    if (rc) return rc;
    const LsDesc<double>& d64 = c.d;
    LsDesc<T> d{};
    d.n_dirs = d64.n_dirs;
    d.nf1 = d64.nf1;
    d.n_pup = d64.n_pup;
    d.n_layers = d64.n_layers;
    d.n_dms = d64.n_dms;
    d.n_a = d64.n_a;
    d.n_slices = d64.n_slices;
    for (int l = 0; l < MAXL; ++l) {
        d.lay_n[l] = d64.lay_n[l];
        d.lay_off[l] = d64.lay_off[l];
    }
    for (int m = 0; m < MAXM; ++m) {
        d.dm_n[m] = d64.dm_n[m];
        d.dm_off[m] = d64.dm_off[m];
    }
    for (int k = 0; k < LSF_MAXK; ++k) d.w[k] = static_cast<T>(d64.w[k]);
    d.eps = static_cast<T>(d64.eps);
    d.mask = d64.mask;
    d.ly0 = d64.ly0;
    d.lx0 = d64.lx0;
    d.my0 = d64.my0;
    d.mx0 = d64.mx0;
    d.ylo = d64.ylo;
    d.yhi = d64.yhi;
    d.xlo = d64.xlo;
    d.xhi = d64.xhi;
    const std::vector<T> lfy(c.L.lfy.begin(), c.L.lfy.end()), lfx(c.L.lfx.begin(), c.L.lfx.end()),
        mfy(c.L.mfy.begin(), c.L.mfy.end()), mfx(c.L.mfx.begin(), c.L.mfx.end());
    d.lfy = lfy.data();
    d.lfx = lfx.data();
    d.mfy = mfy.data();
    d.mfx = mfx.data();
    const int n = d.n_a, npix = d.nf1 * d.nf1, S = d.n_slices, chunk = (npix + S - 1) / S;
    std::vector<T> phi(phi64, phi64 + c.S.n_c), a(n), v(static_cast<size_t>(d.n_dirs) * npix), r(n), p(n), q(n);
    std::vector<double> msum(static_cast<size_t>(d.n_dirs) * S);
    auto sample = [&](const T* src, bool layer) {
        for (int k = 0; k < d.n_dirs; ++k)
            for (int sl = 0; sl < S; ++sl) {
                double acc = 0.0;
                for (int g = sl * chunk; g < std::min(npix, (sl + 1) * chunk); ++g) {
                    T val = T(0);
                    if (d.mask[g]) {
                        const int i = g / d.nf1;
                        val = layer ? lsf_sample<T, true>(d, src, k, i, g - i * d.nf1)
                                    : lsf_sample<T, false>(d, src, k, i, g - i * d.nf1);
                        acc += static_cast<double>(val);
                    }
                    v[static_cast<size_t>(k) * npix + g] = val;
                }
                msum[k * S + sl] = acc;
            }
    };
    auto adjoint = [&](const T* x, T* out) {
        T mean[LSF_MAXK];
        for (int k = 0; k < d.n_dirs; ++k) {
            double t = 0.0;
            for (int sl = 0; sl < S; ++sl) t += msum[k * S + sl];
            mean[k] = static_cast<T>(t / d.n_pup);
        }
        for (int i = 0; i < n; ++i) {
            int m = 0;
            while (m + 1 < d.n_dms && i >= d.dm_off[m + 1]) ++m;
            const int na = d.dm_n[m], loc = i - d.dm_off[m], pp = loc / na;
            T val = lsf_adjoint<T>(d, v.data(), mean, m, pp, loc - pp * na);
            if (x) val += d.eps * x[i];
            out[i] = val;
        }
    };
    sample(phi.data(), true);
    adjoint(nullptr, q.data());
    double rr = 0.0;
    for (int i = 0; i < n; ++i) {
        a[i] = T(0);
        r[i] = p[i] = q[i];
        rr += static_cast<double>(q[i]) * static_cast<double>(q[i]);
    }
    const double rr0 = rr;
    int it = 0;
    bool stop = rr == 0.0 || max_iters <= 0;
    while (!stop) {
        sample(p.data(), false);
        adjoint(p.data(), q.data());
        double pq = 0.0;
        for (int i = 0; i < n; ++i) pq += static_cast<double>(p[i]) * static_cast<double>(q[i]);
        if (!(pq > 0.0)) break;
        const T al = static_cast<T>(rr / pq);
        double rn = 0.0;
        for (int i = 0; i < n; ++i) {
            const T ri = r[i] - al * q[i];
            a[i] += al * p[i];
            r[i] = ri;
            rn += static_cast<double>(ri) * static_cast<double>(ri);
        }
        const T beta = static_cast<T>(rn / rr);
        for (int i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rr = rn;
        ++it;
        if (!(rn > tol * tol * rr0) || it >= max_iters) stop = true;
    }
    for (int i = 0; i < n; ++i) a64[i] = static_cast<double>(a[i]);
    *iters = it;
    *rel = rr0 > 0.0 ? std::sqrt(rr / rr0) : 0.0;
    return 0;
}

}  // namespace

extern "C" int lsfit_host_solve(const fewha_telescope* tel, const fewha_wfs* wfs, int n_wfs,
                                const fewha_layer* layers, int n_layers, const fewha_dm* dms, int n_dms,
                                const fewha_lsfit* cfg, int precision, const double* phi, double* a, double tol,
                                int max_iters, int* iters, double* rel) {
    return precision == 32 ? solve<float>(tel, wfs, n_wfs, layers, n_layers, dms, n_dms, cfg, phi, a, tol,
                                          max_iters, iters, rel)
                           : solve<double>(tel, wfs, n_wfs, layers, n_layers, dms, n_dms, cfg, phi, a, tol,
                                           max_iters, iters, rel);
}
