// mdl_geometry.cpp -- maps of curved meshes and their per-element SIPG factors (host, FP64).
#include "mdl_geometry.h"

#include <math.h>
#include <string.h>

#include <cmath>

#include "mdl_tables.h"

namespace mdl {

GeoArgs geo_args(const mdl_problem& p) {
    GeoArgs g{};
    g.dim = p.dim;
    g.geometry = p.geometry;
    g.fibre_ref = p.fibre_ref;
    for (int k = 0; k < 3; ++k) {
        g.extent[k] = p.extent[k];
        g.iext[k] = p.extent[k] != 0.0 ? 1.0 / p.extent[k] : 0.0;
    }
    for (int i = 0; i < 12; ++i) g.geo[i] = p.geo[i];
    double f0[3] = {p.fibre[0], p.fibre[1], p.dim == 3 ? p.fibre[2] : 0.0};
    double nf0 = 0.0;
    for (int k = 0; k < p.dim; ++k) nf0 += f0[k] * f0[k];
    nf0 = sqrt(nf0);
    for (int k = 0; k < 3; ++k) g.f0[k] = nf0 > 0.0 ? f0[k] / nf0 : (k == 0 ? 1.0 : 0.0);
    g.sig_l = p.sigma_l;
    g.sig_t = p.sigma_t;
    g.chi_cm = p.chi * p.cm;
    g.gamma = p.gamma;
    return g;
}

void geo_map(const mdl_problem& p, const double X[3], double x[3], double J[3][3]) {
    geo_eval(geo_args(p), X, x, J);
}

int geo_check(const mdl_problem& p, const char** why) {
    const int d = p.dim;
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(p.geo[i])) {
            *why = "geo parameters must be finite";
            return MDL_E_ARG;
        }
    if (p.geometry == MDL_GEOMETRY_BOX) return MDL_OK;
    if (p.geometry != MDL_GEOMETRY_AFFINE && p.geometry != MDL_GEOMETRY_SHELL) {
        *why = "geometry must be MDL_GEOMETRY_BOX, _AFFINE or _SHELL";
        return MDL_E_ARG;
    }
    if (p.amr_enabled && !(p.dt_barrier > 0.0)) {
        // an adapting curved mesh has no finite set of element classes to bound the step by
        *why = "a mapped geometry with adaptation needs dt_barrier > 0";
        return MDL_E_ARG;
    }
    if (p.geometry == MDL_GEOMETRY_AFFINE) {
        const double* A = p.geo;
        const double det = d == 2 ? A[0] * A[4] - A[1] * A[3]
                                  : A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                                        A[2] * (A[3] * A[7] - A[4] * A[6]);
        if (!(fabs(det) > 0.0)) {
            *why = "affine geometry: singular matrix";
            return MDL_E_ARG;
        }
        return MDL_OK;
    }
    const double* g = p.geo;
    const int na = d == 2 ? 2 : 3;
    for (int k = 0; k < na; ++k) {
        if (!(g[k] > 0.0) || !(g[3 + k] > 0.0)) {
            *why = "shell geometry: semi-axes must be positive";
            return MDL_E_ARG;
        }
        if (!((g[3 + k] - g[k]) * (g[3] - g[0]) > 0.0)) {
            *why = "shell geometry: every semi-axis must grow (or every one shrink) from inner to outer";
            return MDL_E_ARG;
        }
    }
    if (!(g[7] != 0.0)) {
        *why = "shell geometry: dphi must be nonzero";
        return MDL_E_ARG;
    }
    if (d == 3) {
        const double t1 = g[8] + g[9];
        if (!(g[9] != 0.0) || !(g[8] > 0.0 && g[8] < M_PI) || !(t1 > 0.0 && t1 < M_PI)) {
            *why = "shell geometry: the polar angle range must lie inside (0, pi)";
            return MDL_E_ARG;
        }
    }
    return MDL_OK;
}

namespace {

template <int DIM, int P>
int root_factors(const mdl_problem& p, const Tables<double>& T, MappedFactors* out, std::string* err) {
    constexpr int N1 = P + 1;
    constexpr int NP = DIM == 2 ? N1 * N1 : N1 * N1 * N1, NF = 2 * DIM, NPF = DIM == 2 ? N1 : N1 * N1;
    constexpr int NS = DIM * (DIM + 1) / 2;
    const GeoArgs g = geo_args(p);
    double xg[3], wg[3];
    gl_nodes(P, xg, wg);
    double h0[3] = {1.0, 1.0, 1.0};
    int64_t ne = 1;
    for (int k = 0; k < DIM; ++k) {
        h0[k] = p.extent[k] / p.base[k];
        ne *= p.base[k];
    }
    double slo[MDL_MAX_STIM][3] = {}, shi[MDL_MAX_STIM][3] = {};
    for (int s = 0; s < p.n_stim; ++s)
        for (int k = 0; k < 3; ++k) {
            slo[s][k] = p.stim[s].lo[k] - 1e-12;
            shi[s][k] = p.stim[s].hi[k] + 1e-12;
        }
    out->ne = ne;
    out->np = NP;
    out->nf = NF;
    out->npf = NPF;
    out->ns = NS;
    out->gvol.assign((size_t)ne * NP * (NS + 1), 0.0);
    out->gface.assign((size_t)ne * NF * NPF * (DIM + 2), 0.0);
    out->mass.assign((size_t)ne * NP, 0.0);
    out->cfl.assign(ne, 0.0);
    for (int s = 0; s < MDL_MAX_STIM; ++s) out->smask[s].assign(s < p.n_stim ? ne : 0, 0u);
    std::vector<double> B((size_t)NP * NP);
    for (int64_t e = 0; e < ne; ++e) {
        int cc[3] = {0, 0, 0}, kinds[6] = {0, 0, 0, 0, 0, 0};
        int64_t r = e;
        for (int k = 0; k < DIM; ++k) {
            cc[k] = (int)(r % p.base[k]);
            r /= p.base[k];
        }
        for (int f = 0; f < NF; ++f) {
            const int k = f >> 1, sd = f & 1;
            kinds[f] = (sd ? cc[k] == p.base[k] - 1 : cc[k] == 0) ? 0 : 1;
        }
        uint32_t sm[MDL_MAX_STIM] = {0u, 0u, 0u, 0u};
        const double c = geo_element<DIM, P>(g, T, xg, h0, 0, cc, kinds, p.n_stim, slo, shi,
                                              &out->gvol[(size_t)e * NP * (NS + 1)],
                                              &out->gface[(size_t)e * NF * NPF * (DIM + 2)],
                                              &out->mass[(size_t)e * NP], sm, B.data());
        if (!(c > 0.0) || !std::isfinite(c)) {
            *err = "mapped geometry: singular or degenerate element";
            return MDL_E_ARG;
        }
        out->cfl[e] = c;
        for (int s = 0; s < p.n_stim; ++s) out->smask[s][e] = sm[s];
    }
    return MDL_OK;
}

}  // namespace

int mapped_factors(const mdl_problem& p, const Tables<double>& T, MappedFactors* out, std::string* err) {
    if (p.dim == 2) return p.order == 1 ? root_factors<2, 1>(p, T, out, err) : root_factors<2, 2>(p, T, out, err);
    return p.order == 1 ? root_factors<3, 1>(p, T, out, err) : root_factors<3, 2>(p, T, out, err);
}

}  // namespace mdl
