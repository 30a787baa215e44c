// Host-side geometry set-up of a FEWHA instance: masks, interpolation tables,
// gather ranges for the adjoint operators, the diagonal prior D and the 1-D
// wavelet basis functions used by the exact Jacobi diagonal.
//
// Conventions (the same as the kernels'):
//   aperture node (a, b) of sensor g: x = -D/2 + b d_g, y = -D/2 + a d_g (a = row = y)
//   layer node (i, j): x = (j - n/2) delta, y = (i - n/2) delta, periodic grid n x n
//   sensor g sees layer l at s x + theta h, s = 1 - h/H (LGS, cone effect) or 1 (Sec. 2)
//   a subaperture is active iff obs D/2 <= |centre| <= D/2
#include <cmath>
#include <cstring>
#include <algorithm>

#include "fewha_internal.h"

namespace fewha {

void set_elongation(HostSetup& s, double alpha_eta) {
    for (size_t g = 0; g < s.G.size(); ++g) {
        WfsInfo& W = s.G[g];
        W.el = 0;
        W.el_k = W.el_c = W.el_lx = W.el_ly = W.el_x0 = W.el_d = 0.0;
        W.el_K11 = W.el_K12 = W.el_K22 = 0.0;
        for (float& f : W.el_f) f = 0.f;
        if (!W.lgs || W.nb != 1 || !(alpha_eta > 0) || !(s.wfs_na_fwhm[g] > 0) || !(s.wfs_spot_fwhm[g] > 0))
            continue;
        W.el = 1;
        W.el_k = s.wfs_na_fwhm[g] / (s.wfs_H[g] * s.wfs_H[g]);
        W.el_c = (alpha_eta / s.wfs_spot_fwhm[g]) * (alpha_eta / s.wfs_spot_fwhm[g]);
        W.el_lx = s.wfs_lx[g];
        W.el_ly = s.wfs_ly[g];
        W.el_d = s.D / W.N;
        W.el_x0 = -s.D / 2 + 0.5 * W.el_d;
        for (int i = 0; i < W.N; ++i)
            for (int j = 0; j < W.N; ++j) {
                if (s.sidx[W.mask_off + i * W.N + j] < 0) continue;
                const double b1 = W.el_k * (W.el_x0 + j * W.el_d - W.el_lx);
                const double b2 = W.el_k * (W.el_x0 + i * W.el_d - W.el_ly);
                const double gam = W.el_c / (1.0 + W.el_c * (b1 * b1 + b2 * b2));
                W.el_K11 += gam * b1 * b1;
                W.el_K12 += gam * b1 * b2;
                W.el_K22 += gam * b2 * b2;
            }
        const double c9[9] = {W.el_k, W.el_c, W.el_lx, W.el_ly, W.el_x0, W.el_d, W.el_K11, W.el_K12, W.el_K22};
        for (int q = 0; q < 9; ++q) W.el_f[q] = static_cast<float>(c9[q]);
    }
}

void db3_taps(double h[6], double g[6]) {
    // Daubechies' N = 3 scaling filter in closed form (sum h = sqrt 2), Sec. 3.1.
    const double s10 = std::sqrt(10.0);
    const double r = std::sqrt(5.0 + 2.0 * s10);
    const double q = 16.0 * std::sqrt(2.0);
    h[0] = (1.0 + s10 + r) / q;
    h[1] = (5.0 + s10 + 3.0 * r) / q;
    h[2] = (10.0 - 2.0 * s10 + 2.0 * r) / q;
    h[3] = (10.0 - 2.0 * s10 - 2.0 * r) / q;
    h[4] = (5.0 + s10 - 3.0 * r) / q;
    h[5] = (1.0 + s10 - r) / q;
    // wavelet filter g_k = (-1)^k h_(5-k)
    for (int k = 0; k < 6; ++k) g[k] = ((k & 1) ? -1.0 : 1.0) * h[5 - k];
}

static bool is_pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

static int ilog2(int n) {
    int k = 0;
    while ((1 << k) < n) ++k;
    return k;
}

static bool active(int i, int j, int n, double D, double obs) {
    const double d = D / n;
    const double x = -D / 2 + (j + 0.5) * d, y = -D / 2 + (i + 0.5) * d;
    const double r = std::hypot(x, y);
    return r >= obs * D / 2 && r <= D / 2;
}

// Grid coordinates -> (index, weight); false if the 2-point stencil leaves [0, n-1].
static bool interp(double coord, int n, int& i0, double& f) {
    const double fl = std::floor(coord);
    if (!(fl >= 0.0) || fl + 1.0 > n - 1) return false;
    i0 = static_cast<int>(fl);
    f = coord - fl;
    return true;
}

// Rows a whose stencil {i0[a], i0[a] + 1} contains layer row i form [lo, hi) since i0
// is non-decreasing in a.
static void gather_ranges(const int* i0, int count, int n, int* lo, int* hi) {
    for (int i = 0; i < n; ++i) {
        int a = 0;
        while (a < count && i0[a] + 1 < i) ++a;
        lo[i] = a;
        while (a < count && i0[a] <= i) ++a;
        hi[i] = a;
        if (hi[i] < lo[i]) hi[i] = lo[i];
    }
}

// One periodic 1-D synthesis step on x[0..m) (transpose of the analysis
// a_k = sum_t h_t x_(2k+t mod m), d_k = sum_t g_t x_(2k+t mod m)).
static void synth1d(std::vector<double>& x, int m, const double h[6], const double g[6]) {
    std::vector<double> y(x.begin(), x.begin() + m), o(m, 0.0);
    const int half = m / 2;
    for (int k = 0; k < half; ++k)
        for (int t = 0; t < 6; ++t) o[(2 * k + t) % m] += h[t] * y[k] + g[t] * y[half + k];
    std::copy(o.begin(), o.end(), x.begin());
}

static double fitting_share(double h, const std::vector<double>& dm_h, int m) {
    // Linear altitude split between the two neighbouring DMs; wholly to the nearest
    // DM outside their range.
    std::vector<int> order(dm_h.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = static_cast<int>(k);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return dm_h[a] < dm_h[b]; });
    const int nd = static_cast<int>(order.size());
    std::vector<double> w(nd, 0.0);
    if (h >= dm_h[order[nd - 1]]) {
        w[order[nd - 1]] = 1.0;
    } else if (h <= dm_h[order[0]]) {
        w[order[0]] = 1.0;
    } else {
        int a = 0;
        while (a + 1 < nd && dm_h[order[a + 1]] <= h) ++a;
        const double lo = dm_h[order[a]], hi = dm_h[order[a + 1]];
        const double t = (hi - h) / (hi - lo);
        w[order[a]] += t;
        w[order[a + 1]] += 1.0 - t;
    }
    return w[m];
}

int build_setup(const fewha_telescope& tel, const fewha_wfs* wfs, int n_wfs,
                const fewha_layer* layers, int n_layers, const fewha_dm* dms, int n_dms,
                HostSetup& s, std::string& err) {
    if (n_wfs < 1 || n_layers < 1 || n_dms < 1 || !wfs || !layers || !dms) {
        err = "need at least one sensor, one layer and one DM";
        return FEWHA_ERR_INVALID_ARG;
    }
    if (n_wfs > MAXG || n_layers > MAXL || n_dms > MAXM) {
        err = "too many sensors, layers or DMs";
        return FEWHA_ERR_LIMIT;
    }
    if (!(tel.D > 0) || !(tel.obs >= 0) || !(tel.obs < 1)) {
        err = "telescope diameter must be > 0 and obstruction in [0, 1)";
        return FEWHA_ERR_INVALID_ARG;
    }
    db3_taps(s.taps_h, s.taps_g);
    const double D = tel.D;
    s.D = D;
    // layers
    int off = 0;
    s.max_n = 0;
    for (int l = 0; l < n_layers; ++l) {
        const fewha_layer& L = layers[l];
        if (!is_pow2(L.n)) { err = "layer grid side must be a power of two >= 2"; return FEWHA_ERR_GEOMETRY; }
        if (L.n > MAXN) { err = "layer grid side above FEWHA_MAX_GRID"; return FEWHA_ERR_LIMIT; }
        const int J = ilog2(L.n);
        if (L.levels < 1 || L.levels > J) { err = "wavelet levels out of range"; return FEWHA_ERR_GEOMETRY; }
        if (!(L.spacing > 0) || !(L.cn2_weight > 0) || !(L.h >= 0)) {
            err = "layer spacing and Cn2 weight must be > 0, altitude >= 0";
            return FEWHA_ERR_INVALID_ARG;
        }
        LayerInfo li{L.n, J, L.levels, off, L.levels == J ? 1 : 0};
        s.L.push_back(li);
        s.layer_h.push_back(L.h);
        s.layer_w.push_back(L.cn2_weight);
        s.layer_delta.push_back(L.spacing);
        off += L.n * L.n;
        s.max_n = std::max(s.max_n, L.n);
    }
    s.n_c = off;
    // sensors
    s.pi0y.assign(MAXG * MAXL * TAB, 0);
    s.pi0x.assign(MAXG * MAXL * TAB, 0);
    s.pfy.assign(MAXG * MAXL * TAB, 0.0);
    s.pfx.assign(MAXG * MAXL * TAB, 0.0);
    s.ry_lo.assign(MAXG * MAXL * MAXN, 0);
    s.ry_hi.assign(MAXG * MAXL * MAXN, 0);
    s.rx_lo.assign(MAXG * MAXL * MAXN, 0);
    s.rx_hi.assign(MAXG * MAXL * MAXN, 0);
    int soff = 0, noff = 0, moff = 0, coff = 0;
    s.max_N = 0;
    for (int g = 0; g < n_wfs; ++g) {
        const fewha_wfs& W = wfs[g];
        if (W.n_sub < 1 || W.nb < 1) { err = "n_sub and nb must be >= 1"; return FEWHA_ERR_INVALID_ARG; }
        if (W.is_lgs && W.nb != 1) { err = "an LGS sensor cannot be coarse (nb must be 1)"; return FEWHA_ERR_GEOMETRY; }
        if (W.is_lgs && !(W.H > 0)) { err = "an LGS needs a positive height H"; return FEWHA_ERR_INVALID_ARG; }
        if (!(W.sigma > 0)) { err = "sensor sigma must be > 0"; return FEWHA_ERR_INVALID_ARG; }
        const int N = W.n_sub * W.nb;
        if (N > MAXNF) { err = "n_sub * nb above FEWHA_MAX_NFINE"; return FEWHA_ERR_LIMIT; }
        if (W.nb > 1 && W.n_sub > FEWHA_MAX_COARSE) { err = "coarse sensor above FEWHA_MAX_COARSE"; return FEWHA_ERR_LIMIT; }
        s.max_N = std::max(s.max_N, N);
        WfsInfo wi{};
        wi.N = N;
        wi.nb = W.nb;
        wi.n_sub = W.n_sub;
        wi.lgs = W.is_lgs ? 1 : 0;
        wi.sig2inv = 1.0 / (W.sigma * W.sigma);
        wi.soff = soff;
        wi.node_off = noff;
        wi.mask_off = moff;
        wi.cmask_off = coff;
        // slope index tables
        int count = 0;
        if (W.nb == 1) {
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j)
                    s.sidx.push_back(active(i, j, N, D, tel.obs) ? count++ : -1);
        } else {
            std::vector<int> cid(W.n_sub * W.n_sub, -1);
            for (int I = 0; I < W.n_sub; ++I)
                for (int J = 0; J < W.n_sub; ++J)
                    if (active(I, J, W.n_sub, D, tel.obs)) cid[I * W.n_sub + J] = count++;
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    const int K = cid[(i / W.nb) * W.n_sub + (j / W.nb)];
                    s.sidx.push_back((K >= 0 && active(i, j, N, D, tel.obs)) ? K : -1);
                }
            for (int v : cid) s.cidx.push_back(v);
            coff += W.n_sub * W.n_sub;
        }
        if (count == 0) { err = "a sensor has no active subaperture"; return FEWHA_ERR_GEOMETRY; }
        wi.n_active = count;
        moff += N * N;
        soff += 2 * count;
        noff += (N + 1) * (N + 1);
        // projection tables per layer (Sec. 2: NGS / LGS propagation)
        const double d = D / N;
        for (int l = 0; l < n_layers; ++l) {
            const double h = layers[l].h, delta = layers[l].spacing;
            const int n = layers[l].n;
            const double sc = W.is_lgs ? 1.0 - h / W.H : 1.0;
            if (!(sc > 0)) { err = "layer at or above the LGS height"; return FEWHA_ERR_GEOMETRY; }
            const int base = (g * MAXL + l) * TAB;
            for (int a = 0; a <= N; ++a) {
                const double xa = -D / 2 + a * d;
                int iy, ix;
                double fy, fx;
                if (!interp((sc * xa + W.theta_y * h) / delta + n / 2, n, iy, fy) ||
                    !interp((sc * xa + W.theta_x * h) / delta + n / 2, n, ix, fx)) {
                    err = "sensor footprint leaves the grid of layer " + std::to_string(l);
                    return FEWHA_ERR_GEOMETRY;
                }
                s.pi0y[base + a] = iy;
                s.pfy[base + a] = fy;
                s.pi0x[base + a] = ix;
                s.pfx[base + a] = fx;
            }
            const int rb = (g * MAXL + l) * MAXN;
            gather_ranges(&s.pi0y[base], N + 1, n, &s.ry_lo[rb], &s.ry_hi[rb]);
            gather_ranges(&s.pi0x[base], N + 1, n, &s.rx_lo[rb], &s.rx_hi[rb]);
        }
        s.G.push_back(wi);
        s.wfs_sigma.push_back(W.sigma);
        s.wfs_lx.push_back(W.launch_x);
        s.wfs_ly.push_back(W.launch_y);
        s.wfs_na_fwhm.push_back(W.is_lgs ? W.na_fwhm : 0.0);
        s.wfs_spot_fwhm.push_back(W.is_lgs ? W.spot_fwhm : 0.0);
        s.wfs_H.push_back(W.H);
    }
    s.n_s = soff;
    s.n_nodes = noff;
    // DMs and the fitting split
    std::vector<double> dm_h;
    for (int m = 0; m < n_dms; ++m) dm_h.push_back(dms[m].h);
    s.di0.assign(MAXM * MAXL * MAXNACT, 0);
    s.dfw.assign(MAXM * MAXL * MAXNACT, 0.0);
    s.dr_lo.assign(MAXM * MAXL * MAXN, 0);
    s.dr_hi.assign(MAXM * MAXL * MAXN, 0);
    std::memset(s.fitw, 0, sizeof(s.fitw));
    int aoff = 0;
    for (int m = 0; m < n_dms; ++m) {
        const int na = dms[m].n_act;
        if (na < 1 || na > MAXNACT) { err = "DM actuator count out of range"; return FEWHA_ERR_LIMIT; }
        if (!(dms[m].spacing > 0)) { err = "DM spacing must be > 0"; return FEWHA_ERR_INVALID_ARG; }
        s.Mi.push_back(DmInfo{na, aoff});
        aoff += na * na;
        for (int l = 0; l < n_layers; ++l) {
            const double w = fitting_share(layers[l].h, dm_h, m);
            s.fitw[m][l] = w;
            if (w == 0.0) continue;
            const int base = (m * MAXL + l) * MAXNACT;
            const int n = layers[l].n;
            for (int k = 0; k < na; ++k) {
                const double x = (k - (na - 1) / 2.0) * dms[m].spacing;
                int i0;
                double f;
                if (!interp(x / layers[l].spacing + n / 2, n, i0, f)) {
                    err = "DM " + std::to_string(m) + " leaves the grid of layer " + std::to_string(l);
                    return FEWHA_ERR_GEOMETRY;
                }
                s.di0[base + k] = i0;
                s.dfw[base + k] = f;
            }
            const int rb = (m * MAXL + l) * MAXN;
            gather_ranges(&s.di0[base], na, n, &s.dr_lo[rb], &s.dr_hi[rb]);
        }
    }
    s.n_act = aoff;
    // DM shapes seen by the sensors (closed loop, Algorithm 1): the mirror surface is
    // bilinear between actuators (Sec. 4.1); actuator k of DM m sits at
    // (k - (n_act - 1)/2) spacing; sensor g sees it at s x + theta h_m like a layer
    s.qi0y.assign(MAXG * MAXM * TAB, 0);
    s.qi0x.assign(MAXG * MAXM * TAB, 0);
    s.qfy.assign(MAXG * MAXM * TAB, 0.0);
    s.qfx.assign(MAXG * MAXM * TAB, 0.0);
    for (int g = 0; g < n_wfs; ++g) {
        const fewha_wfs& W = wfs[g];
        const int N = W.n_sub * W.nb;
        const double d = D / N;
        for (int m = 0; m < n_dms; ++m) {
            const double h = dms[m].h, sp = dms[m].spacing, c = (dms[m].n_act - 1) / 2.0;
            const double sc = W.is_lgs ? 1.0 - h / W.H : 1.0;
            if (!(sc > 0)) s.dm_proj_ok = false;
            const int base = (g * MAXM + m) * TAB;
            for (int a = 0; a <= N; ++a) {
                const double xa = -D / 2 + a * d;
                const double uy = (sc * xa + W.theta_y * h) / sp + c, ux = (sc * xa + W.theta_x * h) / sp + c;
                const double fy = std::floor(uy), fx = std::floor(ux);
                // far outside the lattice both stencil points are outside: clamp the index
                s.qi0y[base + a] = static_cast<int>(std::max(-2.0, std::min(fy, double(MAXNACT + 1))));
                s.qfy[base + a] = uy - fy;
                s.qi0x[base + a] = static_cast<int>(std::max(-2.0, std::min(fx, double(MAXNACT + 1))));
                s.qfx[base + a] = ux - fx;
            }
        }
    }
    // 1-D basis functions: synthesis of a unit coefficient of level j through j steps
    s.basis_off.assign(MAXL * (MAXLEV + 1) * 2, -1);
    for (int l = 0; l < n_layers; ++l) {
        const int n = s.L[l].n;
        for (int j = 1; j <= s.L[l].levels; ++j)
            for (int kind = 0; kind < 2; ++kind) {
                std::vector<double> e(n, 0.0);
                e[kind == 0 ? 0 : (n >> j)] = 1.0;
                for (int lev = j - 1; lev >= 0; --lev) synth1d(e, n >> lev, s.taps_h, s.taps_g);
                s.basis_off[basis_index(l, j, kind)] = static_cast<int>(s.basis.size());
                s.basis.insert(s.basis.end(), e.begin(), e.end());
            }
    }
    return FEWHA_OK;
}

// Least-squares fit over fitting directions (Sec. 4.1): pupil node x along direction
// theta sees layer l at x + theta h_l (linear stencils on its grid, which they must not
// leave) and DM m at x + theta h_m (the bilinear hats of its actuators, which are zero
// beyond the outer ones).
int build_lsfit(const HostSetup& s, double obs, const fewha_dm* dms, const fewha_lsfit& cfg,
                LsfitHost& o, std::string& err) {
    const int K = cfg.n_dirs, nf1 = cfg.n_fit + 1;
    const int n_layers = static_cast<int>(s.L.size()), n_dms = static_cast<int>(s.Mi.size());
    const double D = s.D;
    std::vector<double> xs(nf1);
    for (int i = 0; i < nf1; ++i) xs[i] = -D / 2 + i * (D / cfg.n_fit);
    o.n_dirs = K;
    o.nf1 = nf1;
    o.mask.assign(static_cast<size_t>(nf1) * nf1, 0);
    o.n_pup = 0;
    for (int i = 0; i < nf1; ++i)
        for (int j = 0; j < nf1; ++j) {
            const double r = std::hypot(xs[j], xs[i]);
            if (r >= obs * D / 2 && r <= D / 2) {
                o.mask[static_cast<size_t>(i) * nf1 + j] = 1;
                ++o.n_pup;
            }
        }
    if (o.n_pup == 0) { err = "no pupil node of the fitting grid lies in the aperture"; return FEWHA_ERR_GEOMETRY; }
    o.ly0.assign(static_cast<size_t>(K) * MAXL * nf1, 0);
    o.lx0 = o.ly0;
    o.lfy.assign(o.ly0.size(), 0.0);
    o.lfx = o.lfy;
    o.my0.assign(static_cast<size_t>(K) * MAXM * nf1, 0);
    o.mx0 = o.my0;
    o.mfy.assign(o.my0.size(), 0.0);
    o.mfx = o.mfy;
    o.ylo.assign(static_cast<size_t>(K) * MAXM * MAXNACT, 0);
    o.yhi = o.ylo;
    o.xlo = o.ylo;
    o.xhi = o.ylo;
    for (int k = 0; k < K; ++k) {
        const double tx = cfg.theta_x[k], ty = cfg.theta_y[k];
        for (int l = 0; l < n_layers; ++l) {
            const double h = s.layer_h[l], delta = s.layer_delta[l];
            const int n = s.L[l].n;
            const size_t base = (static_cast<size_t>(k) * MAXL + l) * nf1;
            for (int i = 0; i < nf1; ++i) {
                int iy, ix;
                double fy, fx;
                if (!interp((xs[i] + ty * h) / delta + n / 2, n, iy, fy) ||
                    !interp((xs[i] + tx * h) / delta + n / 2, n, ix, fx)) {
                    err = "fitting direction " + std::to_string(k) + " leaves the grid of layer " +
                          std::to_string(l);
                    return FEWHA_ERR_GEOMETRY;
                }
                o.ly0[base + i] = iy;
                o.lfy[base + i] = fy;
                o.lx0[base + i] = ix;
                o.lfx[base + i] = fx;
            }
        }
        for (int m = 0; m < n_dms; ++m) {
            const double h = dms[m].h, sp = dms[m].spacing;
            const int na = dms[m].n_act;
            const size_t base = (static_cast<size_t>(k) * MAXM + m) * nf1;
            for (int i = 0; i < nf1; ++i) {
                const double uy = (xs[i] + ty * h) / sp + (na - 1) / 2.0;
                const double ux = (xs[i] + tx * h) / sp + (na - 1) / 2.0;
                const double fly = std::floor(uy), flx = std::floor(ux);
                // far outside the lattice only the clamp matters: both hats are zero there
                o.my0[base + i] = static_cast<int>(std::max(-2.0, std::min(fly, double(na) + 1.0)));
                o.mfy[base + i] = uy - fly;
                o.mx0[base + i] = static_cast<int>(std::max(-2.0, std::min(flx, double(na) + 1.0)));
                o.mfx[base + i] = ux - flx;
            }
            // pupil rows (columns) i touch actuator row p iff i0[i] is p - 1 or p; i0 is
            // non-decreasing in i, so they form one range
            const size_t rb = (static_cast<size_t>(k) * MAXM + m) * MAXNACT;
            for (int pass = 0; pass < 2; ++pass) {
                const int* i0 = (pass == 0 ? o.my0.data() : o.mx0.data()) + base;
                int* lo = (pass == 0 ? o.ylo.data() : o.xlo.data()) + rb;
                int* hi = (pass == 0 ? o.yhi.data() : o.xhi.data()) + rb;
                for (int p = 0; p < na; ++p) {
                    int a = 0;
                    while (a < nf1 && i0[a] < p - 1) ++a;
                    int b = a;
                    while (b < nf1 && i0[b] <= p) ++b;
                    lo[p] = a;
                    hi[p] = b > a ? b : a;
                }
            }
        }
    }
    return FEWHA_OK;
}

void db3_step_host(double* x, int m, int st, const double* h, const double* g, bool inv) {
    double y[8];
    const int hm = m / 2;
    for (int k = 0; k < hm; ++k) {
        if (!inv) {
            double a = 0.0, d = 0.0;
            for (int t = 0; t < 6; ++t) {
                a += h[t] * x[((2 * k + t) % m) * st];
                d += g[t] * x[((2 * k + t) % m) * st];
            }
            y[k] = a;
            y[hm + k] = d;
        } else {
            double e = 0.0, o = 0.0;
            for (int s2 = 0; s2 < 3; ++s2) {
                const int i = ((k - s2) % hm + hm) % hm;
                e += h[2 * s2] * x[i * st] + g[2 * s2] * x[(hm + i) * st];
                o += h[2 * s2 + 1] * x[i * st] + g[2 * s2 + 1] * x[(hm + i) * st];
            }
            y[2 * k] = e;
            y[2 * k + 1] = o;
        }
    }
    for (int k = 0; k < m; ++k) x[k * st] = y[k];
}

// The tail matrix (rows, then columns, for block sides 8, 4, 2), entry (k, o) at k * ld + o.
// The synthesis of the same steps is checked to be A^T, which the inverse kernel applies;
// empty if not.
std::vector<double> tail_operator(const double* h, const double* g, int ld) {
    std::vector<double> A(static_cast<size_t>(64) * ld, 0.0);
    for (int k = 0; k < 64; ++k) {
        double X[64] = {};
        X[k] = 1.0;
        for (int m = 8; m >= 2; m /= 2) {
            for (int i = 0; i < m; ++i) db3_step_host(X + 8 * i, m, 1, h, g, false);   // rows
            for (int j = 0; j < m; ++j) db3_step_host(X + j, m, 8, h, g, false);       // columns
        }
        for (int o = 0; o < 64; ++o) A[k * ld + o] = X[o];
    }
    for (int o = 0; o < 64; ++o) {
        double Y[64] = {};
        Y[o] = 1.0;
        for (int m = 2; m <= 8; m *= 2) {
            for (int j = 0; j < m; ++j) db3_step_host(Y + j, m, 8, h, g, true);        // columns
            for (int i = 0; i < m; ++i) db3_step_host(Y + 8 * i, m, 1, h, g, true);    // rows
        }
        for (int k = 0; k < 64; ++k)
            if (std::fabs(Y[k] - A[k * ld + o]) > 1e-12) return {};
    }
    return A;
}

// D (Sec. 3.1): a diagonal stand-in for C_phi^-1 on the wavelet coefficients.  For a
// level band (detail level j: FFT index box [-n/2^j, n/2^j)^2 minus [-n/2^(j+1),
// n/2^(j+1))^2; the coarsest approximation: [-n/2^(L+1), n/2^(L+1))^2) the
// coefficient variance is the band mean of (n dk)^2 w Phi(|k| dk), dk = 1/(n delta),
// Phi(f) = 0.023 r0^(-5/3) (f^2 + L0^-2)^(-11/6); D = 1/variance.
void prior_diag(const HostSetup& s, const std::vector<double>& weights, double r0, double L0,
                std::vector<double>& D) {
    D.assign(s.n_c, 0.0);
    for (size_t l = 0; l < s.L.size(); ++l) {
        const int n = s.L[l].n, lev = s.L[l].levels;
        const double dk = 1.0 / (n * s.layer_delta[l]);
        std::vector<double> sum(lev + 2, 0.0);
        std::vector<long> cnt(lev + 2, 0);
        for (int ky = -n / 2; ky < n / 2; ++ky)
            for (int kx = -n / 2; kx < n / 2; ++kx) {
                // band of (ky, kx): the largest j with the index inside [-n/2^j, n/2^j)^2
                int band = 0;
                for (int j = 1; j <= lev + 1; ++j) {
                    const double m = n / std::ldexp(1.0, j);
                    if (ky >= -m && ky < m && kx >= -m && kx < m) band = j;
                }
                // band j >= 1 is "inside box j": it belongs to detail level j unless it
                // is also inside box j+1; box lev+1 is the LL band
                const double f2 = (double(kx) * kx + double(ky) * ky) * dk * dk;
                const double psd = 0.023 * std::pow(r0, -5.0 / 3.0) *
                                   std::pow(f2 + 1.0 / (L0 * L0), -11.0 / 6.0);
                const double var = (n * dk) * (n * dk) * weights[l] * psd;
                sum[band] += var;
                cnt[band] += 1;
            }
        // band index 0 would be outside box 1, impossible for |k| < n/2
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const int mx = std::max(i, j);
                int b;
                if (mx < (n >> lev)) {
                    b = lev + 1;
                } else {
                    b = 1;
                    while (mx < (n >> b)) ++b;   // n>>b <= mx < n>>(b-1)
                }
                D[s.L[l].off + i * n + j] = static_cast<double>(cnt[b]) / sum[b];
            }
    }
}

}  // namespace fewha
