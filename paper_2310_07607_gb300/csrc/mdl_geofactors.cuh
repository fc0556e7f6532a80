// mdl_geofactors.cuh -- the map of a curved mesh and one element's SIPG factors, for the host
// (the root mesh) and the device (after every adaptation): the same code on both.
//
// Element of level l with integer coordinates c: reference box [c h_l, (c + 1) h_l], element
// map x(xi) = Phi(X_c + (xi + 1) h_l / 2), J = DPhi(X) diag(h_l / 2).  Stored per element:
//   volume node q:  G_q = W_q |det DPhi| S DPhi^-1 D(x) DPhi^-T S (S = diag(2/h), W_q = w_q prod h/2),
//                   symmetric (xx, yy, xy | xx, yy, zz, xy, xz, yz), then M_q = W_q |det DPhi|;
//   face point t:   c = S DPhi^-1 D(x) n (n the outward unit normal, along DPhi^-T e_k), the area
//                   weight dS = W_t |det DPhi| |DPhi^-T e_k| and the penalty
//                   kappa = gamma n.D n (1/h_n,own + 1/h_n,nb) / 2 with h_n = h_k / |DPhi^-T e_k|
//                   (h_nb = h_own, 2 h_own or h_own / 2 for a same-level, coarser or finer
//                   neighbour), at the element's own face GL points.
// A face with finer neighbours is integrated on their subfaces (each neighbour holds the
// points, its flux vector, area weight and penalty); here it enters the element's own block
// only, from which the Gershgorin bound CFL_e = 1 / max_i sum_j |B_ij| / M_i
// (Eq. cfl-monodomain) is returned.
#pragma once

#include <math.h>
#include <stdint.h>

#include "../../include/mdl.h"
#include "mdl_element.cuh"

namespace mdl {

// The problem's geometry and diffusion (plain values, for host and device).
struct GeoArgs {
    int dim, geometry, fibre_ref;
    double extent[3];
    double iext[3];           // 1 / extent
    double geo[12];
    double f0[3];             // normalised fibre (fibre_ref = 0)
    double sig_l, sig_t, chi_cm, gamma;
};

// sin and cos of one angle (the device computes both from one argument reduction).
MDL_HD void geo_sincos(double a, double* s, double* c) {
#ifdef __CUDA_ARCH__
    sincos(a, s, c);
#else
    *s = sin(a);
    *c = cos(a);
#endif
}

// x = Phi(X) and J = DPhi(X) (J[i][j] = d x_i / d X_j), 3D layout (2D: leading 2 x 2 block).
MDL_HD void geo_eval(const GeoArgs& g, const double X[3], double x[3], double J[3][3]) {
    for (int i = 0; i < 3; ++i) {
        x[i] = X[i];
        for (int j = 0; j < 3; ++j) J[i][j] = i == j ? 1.0 : 0.0;
    }
    const int d = g.dim;
    const double* p = g.geo;
    if (g.geometry == MDL_GEOMETRY_AFFINE) {
        for (int i = 0; i < d; ++i) {
            x[i] = p[9 + i];
            for (int j = 0; j < d; ++j) {
                x[i] += p[3 * i + j] * X[j];
                J[i][j] = p[3 * i + j];
            }
        }
        return;
    }
    if (g.geometry != MDL_GEOMETRY_SHELL) return;
    const double ai = p[0], bi = p[1], ci = p[2], ao = p[3], bo = p[4], co = p[5];
    const double p0 = p[6], dp = p[7], t0 = p[8], dt = p[9];
    // (products by the inverse extents: FP64 division is a long instruction sequence)
    const double e0 = g.iext[0], e1 = g.iext[1], e2 = g.iext[2];
    const double az = p0 + X[0] * e0 * dp;
    double sp, cp;
    geo_sincos(az, &sp, &cp);
    if (d == 2) {
        const double u = X[1] * e1;
        const double a = ai + u * (ao - ai), b = bi + u * (bo - bi);
        x[0] = a * cp;
        x[1] = b * sp;
        J[0][0] = -a * sp * dp * e0;
        J[1][0] = b * cp * dp * e0;
        J[0][1] = (ao - ai) * cp * e1;
        J[1][1] = (bo - bi) * sp * e1;
        return;
    }
    const double th = t0 + X[1] * e1 * dt;
    double st, ct;
    geo_sincos(th, &st, &ct);
    const double u = X[2] * e2;
    const double a = ai + u * (ao - ai), b = bi + u * (bo - bi), c = ci + u * (co - ci);
    x[0] = a * st * cp;
    x[1] = b * st * sp;
    x[2] = c * ct;
    J[0][0] = -a * st * sp * dp * e0;
    J[1][0] = b * st * cp * dp * e0;
    J[2][0] = 0.0;
    J[0][1] = a * ct * cp * dt * e1;
    J[1][1] = b * ct * sp * dt * e1;
    J[2][1] = -c * st * dt * e1;
    J[0][2] = (ao - ai) * st * cp * e2;
    J[1][2] = (bo - bi) * st * sp * e2;
    J[2][2] = (co - ci) * ct * e2;
}

// Inverse and determinant of the leading d x d block.
MDL_HD double geo_inverse(int d, const double J[3][3], double Ji[3][3]) {
    if (d == 2) {
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double id = 1.0 / det;
        Ji[0][0] = J[1][1] * id;
        Ji[0][1] = -J[0][1] * id;
        Ji[1][0] = -J[1][0] * id;
        Ji[1][1] = J[0][0] * id;
        return det;
    }
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const double id = 1.0 / det;
    Ji[0][0] = c00 * id;
    Ji[1][0] = c01 * id;
    Ji[2][0] = c02 * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    return det;
}

// D(x) = (sigma_t I + (sigma_l - sigma_t) f f^T) / (chi C_m), f constant or along DPhi e_0.
MDL_HD void geo_tensor(const GeoArgs& g, const double J[3][3], double D[3][3]) {
    const int d = g.dim;
    double f[3] = {g.f0[0], g.f0[1], g.f0[2]};
    if (g.fibre_ref) {
        double l = 0.0;
        for (int i = 0; i < d; ++i) l += J[i][0] * J[i][0];
        l = sqrt(l);
        for (int i = 0; i < 3; ++i) f[i] = i < d ? J[i][0] / l : 0.0;
    }
    const double ic = 1.0 / g.chi_cm;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[i][j] = ((i == j ? g.sig_t : 0.0) + (g.sig_l - g.sig_t) * f[i] * f[j]) * ic;
}

// The 1D Lagrange basis of the (p+1) GL nodes xg at t, and its derivative.
template <int N1>
MDL_HD void geo_lagrange(const double* xg, double t, double* l, double* dl) {
    for (int j = 0; j < N1; ++j) {
        double v = 1.0, dv = 0.0;
        for (int m = 0; m < N1; ++m) {
            if (m == j) continue;
            double term = 1.0 / (xg[j] - xg[m]);
            for (int n = 0; n < N1; ++n)
                if (n != j && n != m) term *= (t - xg[n]) / (xg[j] - xg[n]);
            dv += term;
            v *= (t - xg[m]) / (xg[j] - xg[m]);
        }
        l[j] = v;
        dl[j] = dv;
    }
}

// The physical normal data at reference point X of a normal-k face of an element of extents h:
// c = S DPhi^-1 D n (n = sgn DPhi^-T e_k / |.|), |det DPhi|, |DPhi^-T e_k| and n.D n.
MDL_HD void geo_face_point(const GeoArgs& g, const double X[3], const double* h, int k, double sgn, double* c,
                           double* adet, double* ln, double* nDn) {
    const int d = g.dim;
    double x[3], J[3][3], Ji[3][3], D[3][3];
    geo_eval(g, X, x, J);
    const double det = geo_inverse(d, J, Ji);
    geo_tensor(g, J, D);
    double m[3] = {0.0, 0.0, 0.0}, l2 = 0.0;
    for (int i = 0; i < d; ++i) {
        m[i] = Ji[k][i];
        l2 += m[i] * m[i];
    }
    const double l = sqrt(l2), il = 1.0 / l;
    double n[3] = {0.0, 0.0, 0.0}, Dn[3] = {0.0, 0.0, 0.0}, q = 0.0;
    for (int i = 0; i < d; ++i) n[i] = sgn * m[i] * il;
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j < d; ++j) Dn[i] += D[i][j] * n[j];
        q += n[i] * Dn[i];
    }
    for (int i = 0; i < d; ++i) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) s += Ji[i][j] * Dn[j];
        c[i] = s * (2.0 / h[i]);
    }
    *adet = fabs(det);
    *ln = l;
    *nDn = q;
}

// Factors of one element (level lev, integer coordinates cc, face kinds kinds[f]: 0 boundary,
// 1 same level, 2 coarser neighbour, 3 finer neighbours), its GL masses, the stimulus node
// masks of the boxes sb (physical coordinates, slack applied) and, returned, its Gershgorin
// bound; B is NP x NP scratch.  h0 = element extents at level 0.
template <int DIM, int P>
MDL_HD double geo_element(const GeoArgs& g, const Tables<double>& T, const double* xg, const double* h0, int lev,
                          const int* cc, const int* kinds, int nstim, const double (*slo)[3], const double (*shi)[3],
                          double* gvol, double* gface, double* mass, uint32_t* smask, double* B) {
    constexpr int N1 = P + 1;
    constexpr int NP = DIM == 2 ? N1 * N1 : N1 * N1 * N1, NF = 2 * DIM, NPF = DIM == 2 ? N1 : N1 * N1;
    constexpr int NS = DIM * (DIM + 1) / 2, VPN = NS + 1, FPV = DIM + 2;
    double h[3] = {1.0, 1.0, 1.0}, Xc[3] = {0.0, 0.0, 0.0}, s2h[3] = {2.0, 2.0, 2.0};
    const double sc = 1.0 / (double)(1 << lev);
    for (int k = 0; k < DIM; ++k) {
        h[k] = h0[k] * sc;
        Xc[k] = cc[k] * h[k];
        s2h[k] = 2.0 / h[k];
    }
    for (int i = 0; i < NP * NP; ++i) B[i] = 0.0;
    for (int s = 0; s < nstim; ++s) smask[s] = 0u;
    // volume nodes
    for (int q = 0; q < NP; ++q) {
        double X[3] = {0.0, 0.0, 0.0}, x[3], J[3][3], Ji[3][3], D[3][3];
        double W = 1.0;
        for (int k = 0; k < DIM; ++k) {
            const int a = digit<N1>(q, k);
            X[k] = Xc[k] + (xg[a] + 1.0) * 0.5 * h[k];
            W *= T.w[a] * h[k] * 0.5;
        }
        geo_eval(g, X, x, J);
        const double det = geo_inverse(DIM, J, Ji);
        geo_tensor(g, J, D);
        double K[3][3];
        for (int i = 0; i < DIM; ++i)
            for (int j = 0; j < DIM; ++j) {
                double s = 0.0;
                for (int a = 0; a < DIM; ++a)
                    for (int b = 0; b < DIM; ++b) s += Ji[i][a] * D[a][b] * Ji[j][b];
                K[i][j] = W * fabs(det) * s2h[i] * s * s2h[j];
            }
        double* gv = gvol + q * VPN;
        if (DIM == 2) {
            gv[0] = K[0][0]; gv[1] = K[1][1]; gv[2] = K[0][1];
        } else {
            gv[0] = K[0][0]; gv[1] = K[1][1]; gv[2] = K[2][2];
            gv[3] = K[0][1]; gv[4] = K[0][2]; gv[5] = K[1][2];
        }
        mass[q] = W * fabs(det);
        gv[NS] = mass[q];
        for (int s = 0; s < nstim; ++s) {
            bool in = true;
            for (int k = 0; k < DIM; ++k) in = in && x[k] >= slo[s][k] && x[k] <= shi[s][k];
            if (in) smask[s] |= 1u << q;
        }
        // own block, volume: d_k psi_i at node q is D1[a_k(q)][a_k(i)] when q and i differ in digit k only
        for (int k = 0; k < DIM; ++k)
            for (int l = 0; l < DIM; ++l)
                for (int m = 0; m < N1; ++m) {
                    const int i = q + (m - digit<N1>(q, k)) * stride<N1>(k);
                    const double di = T.D1[digit<N1>(q, k)][m] * K[k][l];
                    for (int m2 = 0; m2 < N1; ++m2) {
                        const int j = q + (m2 - digit<N1>(q, l)) * stride<N1>(l);
                        B[i * NP + j] += di * T.D1[digit<N1>(q, l)][m2];
                    }
                }
    }
    // faces
    for (int f = 0; f < NF; ++f) {
        const int k = f >> 1, sd = f & 1, kind = kinds[f];
        const double sgn = sd ? 1.0 : -1.0;
        int tg[2] = {0, 0}, nt = 0;
        for (int l = 0; l < DIM; ++l)
            if (l != k) tg[nt++] = l;
        const double* bs = sd ? T.bR : T.bL;
        const double* ds = sd ? T.dR : T.dL;
        const double pen = kind == 2 ? 0.75 : (kind == 3 ? 1.5 : 1.0);   // (1 + h_own / h_nb) / 2
        const int nsub = kind == 3 ? (1 << (DIM - 1)) : 1;
        for (int sb = 0; sb < nsub; ++sb) {
            for (int t = 0; t < NPF; ++t) {
                const int at[2] = {t % N1, t / N1};
                double X[3] = {0.0, 0.0, 0.0};
                double Wt = 1.0;
                double xi_t[2] = {0.0, 0.0};          // own reference coordinate of the point
                X[k] = Xc[k] + (sd ? h[k] : 0.0);
                for (int z = 0; z < nt; ++z) {
                    const int l = tg[z];
                    if (kind == 3) {
                        // the finer neighbour's GL point on subface sb (half b of the own face)
                        const int bit = (sb >> z) & 1;
                        const double xf = (xg[at[z]] + 2.0 * bit - 1.0) * 0.5;
                        X[l] = Xc[l] + (xf + 1.0) * 0.5 * h[l];
                        Wt *= T.w[at[z]] * h[l] * 0.25;
                        xi_t[z] = xf;
                    } else {
                        X[l] = Xc[l] + (xg[at[z]] + 1.0) * 0.5 * h[l];
                        Wt *= T.w[at[z]] * h[l] * 0.5;
                        xi_t[z] = xg[at[z]];
                    }
                }
                double c[3] = {0.0, 0.0, 0.0}, adet = 0.0, ln = 0.0, nDn = 0.0;
                if (kind != 0) geo_face_point(g, X, h, k, sgn, c, &adet, &ln, &nDn);
                const double dS = Wt * adet * ln;
                const double kap = g.gamma * nDn * ln / h[k] * pen;
                if (sb == 0) {
                    double* gf = gface + (f * NPF + t) * FPV;
                    for (int i = 0; i < FPV; ++i) gf[i] = 0.0;
                    if (kind == 1 || kind == 2) {
                        for (int i = 0; i < DIM; ++i) gf[i] = c[i];
                        gf[DIM] = dS;
                        gf[DIM + 1] = kap;
                    }
                }
                if (kind == 0) continue;
                // own-side quadrant: psi_i and c . grad_xi psi_i at the point
                double lt[2][3], dlt[2][3];
                for (int z = 0; z < nt; ++z) geo_lagrange<N1>(xg, xi_t[z], lt[z], dlt[z]);
                double psi[NP], cg[NP];
                for (int i = 0; i < NP; ++i) {
                    const int ak = digit<N1>(i, k);
                    double tv = 1.0;                  // tangential product of the basis at the point
                    for (int z = 0; z < nt; ++z) tv *= lt[z][digit<N1>(i, tg[z])];
                    psi[i] = bs[ak] * tv;
                    double cgi = c[k] * ds[ak] * tv;
                    for (int z = 0; z < nt; ++z) {
                        double dz = bs[ak] * dlt[z][digit<N1>(i, tg[z])];
                        for (int z2 = 0; z2 < nt; ++z2)
                            if (z2 != z) dz *= lt[z2][digit<N1>(i, tg[z2])];
                        cgi += c[tg[z]] * dz;
                    }
                    cg[i] = cgi;
                }
                for (int i = 0; i < NP; ++i) {
                    if (psi[i] == 0.0 && cg[i] == 0.0) continue;
                    for (int j = 0; j < NP; ++j)
                        B[i * NP + j] += dS * (-0.5 * cg[j] * psi[i] - 0.5 * cg[i] * psi[j] + kap * psi[i] * psi[j]);
                }
            }
        }
    }
    double mx = 0.0;
    for (int i = 0; i < NP; ++i) {
        double row = 0.0;
        for (int j = 0; j < NP; ++j) row += fabs(B[i * NP + j]);
        row /= mass[i];
        mx = row > mx ? row : mx;
    }
    return 1.0 / mx;
}

}  // namespace mdl
