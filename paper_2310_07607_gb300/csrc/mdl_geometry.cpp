// mdl_geometry.cpp -- maps of curved meshes and their per-element SIPG factors (host, FP64).
#include "mdl_geometry.h"

#include <math.h>
#include <string.h>

#include <cmath>

#include "mdl_tables.h"

namespace mdl {

void geo_map(const mdl_problem& p, const double X[3], double x[3], double J[3][3]) {
    for (int i = 0; i < 3; ++i) {
        x[i] = X[i];
        for (int j = 0; j < 3; ++j) J[i][j] = i == j ? 1.0 : 0.0;
    }
    const int d = p.dim;
    const double* g = p.geo;
    if (p.geometry == MDL_GEOMETRY_AFFINE) {
        for (int i = 0; i < d; ++i) {
            x[i] = g[9 + i];
            for (int j = 0; j < d; ++j) {
                x[i] += g[3 * i + j] * X[j];
                J[i][j] = g[3 * i + j];
            }
        }
        return;
    }
    if (p.geometry != MDL_GEOMETRY_SHELL) return;
    const double ai = g[0], bi = g[1], ci = g[2], ao = g[3], bo = g[4], co = g[5];
    const double p0 = g[6], dp = g[7], t0 = g[8], dt = g[9];
    const double az = p0 + X[0] / p.extent[0] * dp;
    const double sp = sin(az), cp = cos(az);
    if (d == 2) {
        const double u = X[1] / p.extent[1];
        const double a = ai + u * (ao - ai), b = bi + u * (bo - bi);
        x[0] = a * cp;
        x[1] = b * sp;
        J[0][0] = -a * sp * dp / p.extent[0];
        J[1][0] = b * cp * dp / p.extent[0];
        J[0][1] = (ao - ai) * cp / p.extent[1];
        J[1][1] = (bo - bi) * sp / p.extent[1];
        return;
    }
    const double th = t0 + X[1] / p.extent[1] * dt;
    const double st = sin(th), ct = cos(th);
    const double u = X[2] / p.extent[2];
    const double a = ai + u * (ao - ai), b = bi + u * (bo - bi), c = ci + u * (co - ci);
    x[0] = a * st * cp;
    x[1] = b * st * sp;
    x[2] = c * ct;
    J[0][0] = -a * st * sp * dp / p.extent[0];
    J[1][0] = b * st * cp * dp / p.extent[0];
    J[2][0] = 0.0;
    J[0][1] = a * ct * cp * dt / p.extent[1];
    J[1][1] = b * ct * sp * dt / p.extent[1];
    J[2][1] = -c * st * dt / p.extent[1];
    J[0][2] = (ao - ai) * st * cp / p.extent[2];
    J[1][2] = (bo - bi) * st * sp / p.extent[2];
    J[2][2] = (co - ci) * ct / p.extent[2];
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
    if (p.amr_enabled || p.max_refine != 0) {
        *why = "a mapped geometry needs amr_enabled = 0 and max_refine = 0 (a fixed root mesh)";
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

// Inverse and determinant of the leading d x d block.
double inverse(int d, const double J[3][3], double Ji[3][3]) {
    if (d == 2) {
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det;
        Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det;
        Ji[1][1] = J[0][0] / det;
        return det;
    }
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    Ji[0][0] = c00 / det;
    Ji[1][0] = c01 / det;
    Ji[2][0] = c02 / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    return det;
}

int dig(int q, int k, int n1) { return k == 0 ? q % n1 : (k == 1 ? (q / n1) % n1 : q / (n1 * n1)); }
int strd(int k, int n1) { return k == 0 ? 1 : (k == 1 ? n1 : n1 * n1); }

}  // namespace

int mapped_factors(const mdl_problem& p, const Tables<double>& T, MappedFactors* out, std::string* err) {
    const int d = p.dim, n1 = p.order + 1;
    const int np = d == 2 ? n1 * n1 : n1 * n1 * n1, nf = 2 * d, npf = d == 2 ? n1 : n1 * n1;
    const int ns = d * (d + 1) / 2;
    double xg[3], wg[3];
    gl_nodes(p.order, xg, wg);
    double h[3] = {1.0, 1.0, 1.0};
    int64_t ne = 1;
    for (int k = 0; k < d; ++k) {
        h[k] = p.extent[k] / p.base[k];
        ne *= p.base[k];
    }
    double f0[3] = {p.fibre[0], p.fibre[1], d == 3 ? p.fibre[2] : 0.0};
    double nf0 = 0.0;
    for (int k = 0; k < d; ++k) nf0 += f0[k] * f0[k];
    nf0 = sqrt(nf0);
    for (int k = 0; k < 3; ++k) f0[k] = nf0 > 0.0 ? f0[k] / nf0 : (k == 0 ? 1.0 : 0.0);
    const double cm = p.chi * p.cm;
    // D(x) = (sigma_t I + (sigma_l - sigma_t) f f^T) / (chi C_m), f constant or along DPhi e_0
    auto tensor = [&](const double J[3][3], double D[3][3]) {
        double f[3] = {f0[0], f0[1], f0[2]};
        if (p.fibre_ref) {
            double l = 0.0;
            for (int i = 0; i < d; ++i) l += J[i][0] * J[i][0];
            l = sqrt(l);
            for (int i = 0; i < 3; ++i) f[i] = i < d ? J[i][0] / l : 0.0;
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                D[i][j] = ((i == j ? p.sigma_t : 0.0) + (p.sigma_l - p.sigma_t) * f[i] * f[j]) / cm;
    };
    out->ne = ne;
    out->np = np;
    out->nf = nf;
    out->npf = npf;
    out->ns = ns;
    out->gvol.assign((size_t)ne * np * (ns + 1), 0.0);
    out->gface.assign((size_t)ne * nf * npf * (d + 2), 0.0);
    out->mass.assign((size_t)ne * np, 0.0);
    out->cfl.assign(ne, 0.0);
    for (int s = 0; s < MDL_MAX_STIM; ++s) out->smask[s].assign(s < p.n_stim ? ne : 0, 0u);
    std::vector<double> B((size_t)np * np), G((size_t)np * 9);
    std::vector<double> psi(np), cg(np);
    for (int64_t e = 0; e < ne; ++e) {
        int ic[3] = {0, 0, 0};
        int64_t r = e;
        for (int k = 0; k < d; ++k) {
            ic[k] = (int)(r % p.base[k]);
            r /= p.base[k];
        }
        double Xc[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < d; ++k) Xc[k] = ic[k] * h[k];
        std::fill(B.begin(), B.end(), 0.0);
        // volume nodes: metric, mass, stimulus masks
        for (int q = 0; q < np; ++q) {
            double X[3] = {0.0, 0.0, 0.0}, x[3], J[3][3], Ji[3][3], D[3][3];
            double W = 1.0;
            for (int k = 0; k < d; ++k) {
                const int a = dig(q, k, n1);
                X[k] = Xc[k] + (xg[a] + 1.0) * 0.5 * h[k];
                W *= wg[a] * h[k] * 0.5;
            }
            geo_map(p, X, x, J);
            const double det = inverse(d, J, Ji);
            if (!(fabs(det) > 0.0) || !std::isfinite(det)) {
                *err = "mapped geometry: singular Jacobian at a node";
                return MDL_E_ARG;
            }
            tensor(J, D);
            double K[3][3];
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    double s = 0.0;
                    for (int a = 0; a < d; ++a)
                        for (int b = 0; b < d; ++b) s += Ji[i][a] * D[a][b] * Ji[j][b];
                    K[i][j] = W * fabs(det) * (2.0 / h[i]) * s * (2.0 / h[j]);
                }
            double* gv = &out->gvol[((size_t)e * np + q) * (ns + 1)];
            if (d == 2) {
                gv[0] = K[0][0]; gv[1] = K[1][1]; gv[2] = K[0][1];
            } else {
                gv[0] = K[0][0]; gv[1] = K[1][1]; gv[2] = K[2][2];
                gv[3] = K[0][1]; gv[4] = K[0][2]; gv[5] = K[1][2];
            }
            const double M = W * fabs(det);
            gv[ns] = M;
            out->mass[(size_t)e * np + q] = M;
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) G[(size_t)q * 9 + i * 3 + j] = K[i][j];
            for (int s = 0; s < p.n_stim; ++s) {
                bool in = true;
                for (int k = 0; k < d; ++k)
                    in = in && x[k] >= p.stim[s].lo[k] - 1e-12 && x[k] <= p.stim[s].hi[k] + 1e-12;
                if (in) out->smask[s][e] |= 1u << q;
            }
        }
        // own block, volume: d_k psi_i at node q is D1[a_k(q)][a_k(i)] when q and i differ
        // in digit k only
        for (int q = 0; q < np; ++q)
            for (int k = 0; k < d; ++k)
                for (int l = 0; l < d; ++l) {
                    const double g = G[(size_t)q * 9 + k * 3 + l];
                    for (int m = 0; m < n1; ++m) {
                        const int i = q + (m - dig(q, k, n1)) * strd(k, n1);
                        const double di = T.D1[dig(q, k, n1)][m];
                        for (int m2 = 0; m2 < n1; ++m2) {
                            const int j = q + (m2 - dig(q, l, n1)) * strd(l, n1);
                            B[(size_t)i * np + j] += di * g * T.D1[dig(q, l, n1)][m2];
                        }
                    }
                }
        // faces
        for (int f = 0; f < nf; ++f) {
            const int k = f >> 1, s = f & 1;
            const bool bnd = s ? ic[k] == p.base[k] - 1 : ic[k] == 0;
            int tg[2] = {0, 0}, nt = 0;
            for (int l = 0; l < d; ++l)
                if (l != k) tg[nt++] = l;
            const double* bs = s ? T.bR : T.bL;
            const double* ds = s ? T.dR : T.dL;
            for (int t = 0; t < npf; ++t) {
                const int at[2] = {t % n1, t / n1};
                double X[3] = {0.0, 0.0, 0.0}, x[3], J[3][3], Ji[3][3], D[3][3];
                double Wt = 1.0;
                X[k] = Xc[k] + (s ? h[k] : 0.0);
                for (int z = 0; z < nt; ++z) {
                    X[tg[z]] = Xc[tg[z]] + (xg[at[z]] + 1.0) * 0.5 * h[tg[z]];
                    Wt *= wg[at[z]] * h[tg[z]] * 0.5;
                }
                if (bnd) continue;
                geo_map(p, X, x, J);
                const double det = inverse(d, J, Ji);
                if (!(fabs(det) > 0.0) || !std::isfinite(det)) {
                    *err = "mapped geometry: singular Jacobian at a face point";
                    return MDL_E_ARG;
                }
                tensor(J, D);
                // DPhi^-T e_k is row k of DPhi^-1
                double m[3] = {0.0, 0.0, 0.0}, ln = 0.0;
                for (int i = 0; i < d; ++i) {
                    m[i] = Ji[k][i];
                    ln += m[i] * m[i];
                }
                ln = sqrt(ln);
                double n[3], Dn[3], c[3], nDn = 0.0;
                for (int i = 0; i < d; ++i) n[i] = (s ? 1.0 : -1.0) * m[i] / ln;
                for (int i = 0; i < d; ++i) {
                    Dn[i] = 0.0;
                    for (int j = 0; j < d; ++j) Dn[i] += D[i][j] * n[j];
                    nDn += n[i] * Dn[i];
                }
                for (int i = 0; i < d; ++i) {
                    c[i] = 0.0;
                    for (int j = 0; j < d; ++j) c[i] += Ji[i][j] * Dn[j];
                    c[i] *= 2.0 / h[i];
                }
                const double dS = Wt * fabs(det) * ln;
                const double kap = p.gamma * nDn * ln / h[k];
                double* gf = &out->gface[(((size_t)e * nf + f) * npf + t) * (d + 2)];
                for (int i = 0; i < d; ++i) gf[i] = c[i];
                gf[d] = dS;
                gf[d + 1] = kap;
                // own-side quadrant of the face block: psi_i and c . grad_xi psi_i at point t
                std::fill(psi.begin(), psi.end(), 0.0);
                std::fill(cg.begin(), cg.end(), 0.0);
                int base_q = 0;
                for (int z = 0; z < nt; ++z) base_q += at[z] * strd(tg[z], n1);
                for (int mm = 0; mm < n1; ++mm) {
                    const int i = base_q + mm * strd(k, n1);
                    psi[i] = bs[mm];
                    cg[i] += c[k] * ds[mm];
                    for (int z = 0; z < nt; ++z)
                        for (int a = 0; a < n1; ++a) {
                            const int i2 = i + (a - at[z]) * strd(tg[z], n1);
                            cg[i2] += c[tg[z]] * bs[mm] * T.D1[at[z]][a];
                        }
                }
                for (int i = 0; i < np; ++i)
                    for (int j = 0; j < np; ++j)
                        B[(size_t)i * np + j] +=
                            dS * (-0.5 * cg[j] * psi[i] - 0.5 * cg[i] * psi[j] + kap * psi[i] * psi[j]);
            }
        }
        // Gershgorin bound of M^-1 B (Eq. cfl-monodomain)
        double mx = 0.0;
        for (int i = 0; i < np; ++i) {
            double row = 0.0;
            for (int j = 0; j < np; ++j) row += fabs(B[(size_t)i * np + j]);
            row /= out->mass[(size_t)e * np + i];
            mx = row > mx ? row : mx;
        }
        out->cfl[e] = 1.0 / mx;
    }
    return MDL_OK;
}

}  // namespace mdl
