// mdl_element.cuh -- matrix-free SIPG element operator on GL-collocated box elements.
//
// One element's residual r = (A u)_e of the symmetric interior penalty form
// (Eq. monodomain-primal-formulation with the anisotropic flux of
// Eq. monodomain-numerical-flux, standard SIPG signs):
//
//   a(u, v) = sum_e int_e D grad u . grad v
//           - sum_F int_F ( {D grad u}.[v] + {D grad v}.[u] ) + sum_F int_F kappa_F [u].[v]
//   kappa_F = gamma (n.D n / h_own + n.D n / h_nb) / 2,   h = element extent normal to F,
//
// evaluated from the element's own side with its outward normal n = s e_k:
//   volume  : sum_k (2/h_k) D1_k^T [ W * sum_l D_kl (2/h_l) D1_l u ]          (sum factorisation)
//   face    : at each face point t with weight W_t,
//               jump = u_own - u_nb,  favg = (n.D grad u_own + n.D grad u_nb) / 2
//               r += psi(x_t) W_t (kappa jump - favg) - 1/2 W_t jump (n.D grad psi)(x_t).
// Hanging faces (2:1) are integrated per fine subface with the fine GL rule; the
// coarse side is evaluated at the mapped points through the 1D interpolation
// matrices Pi[c] (values) and Pd[c] (derivatives) of the half c of its face.
//
// Shared by the CUDA sweep kernels and by the host (FP64) computation of the
// element classes' own blocks for the Gershgorin CFL bound (Eq. cfl-monodomain).
#pragma once

#include <math.h>
#include <stdint.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

#define MDL_HD __host__ __device__ __forceinline__

namespace mdl {

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <int DIM, int P>
struct Shape {
    static constexpr int N1 = P + 1;                 // nodes per direction
    static constexpr int NP = ipow(N1, DIM);         // DOFs per element
    static constexpr int NF = 2 * DIM;               // faces
    static constexpr int NT = ipow(N1, DIM - 1);     // points per (sub)face
    static constexpr int NSUB = 1 << (DIM - 1);      // subfaces of a hanging face
    // Row stride of the per-DOF state arrays (V slots, v, Ia, ga) in device memory: the DOF
    // count, except Q2 3D, whose 27 values are padded to 28 so that every element row starts
    // on a 16-byte boundary (vector loads, bulk copies of whole rows).  The pad is kept 0.
    static constexpr int NPS = (DIM == 3 && P == 2) ? 28 : NP;
};

// 1D tables of the (P+1)-point Gauss-Legendre Lagrange basis (P <= 2), filled on the host.
template <typename R>
struct Tables {
    R D1[3][3];        // D1[i][j] = l_j'(x_i)
    R bL[3], bR[3];    // l_j(-1), l_j(+1)
    R dL[3], dR[3];    // l_j'(-1), l_j'(+1)
    R Pi[2][3][3];     // Pi[c][i][m] = l_m((x_i + 2c - 1)/2): half c of [-1,1]
    R Pd[2][3][3];     // Pd[c][i][m] = l_m'((x_i + 2c - 1)/2)  (d/dx of the coarse reference coord)
    R w[3];            // GL weights
    R pphi[8][3][3];   // probes: pphi[l][a][j] = l_j(rho) with rho the leaf coordinate of root node a at level l
    int32_t pfl[8][3]; // floor((x_a + 1)/2 * 2^l): which level-l cell of the root holds root node a
};

// Geometry and physics of one problem.
template <typename R>
struct Phys {
    R D[3][3];         // diffusion tensor D = kappa / (chi C_m)
    R gamma;
    R h[8][3];         // element extents per level
    R h2[8][3];        // 2 / h
    R Wvol[8];         // prod_k h_k / 2
    R Wface[8][3];     // prod_{l != k} h_l / 2  (face Jacobian of a normal-k face)
    double kfac[8][3]; // h_F / (2p) W_F^2 of a normal-k (sub)face whose finer side has level l
    R Minv[8][27];     // inverse diagonal GL mass 1 / (Wvol prod_k w_{a_k}) per level and node
    // Aliev-Panfilov
    R k, a, eps0, mu1, mu2, inv_ts;
    int32_t ionic;     // 0 AP, -1 none
    int32_t integrator;// 0 FE, 1 exponential
    R act;             // activation threshold
    R lat_gate;        // max|V| below which no probe of the element can exceed act
};

// Tensor digit helpers: q = a0 + N1 a1 + N1^2 a2.
template <int N1>
MDL_HD int digit(int q, int k) { return k == 0 ? q % N1 : (k == 1 ? (q / N1) % N1 : q / (N1 * N1)); }
template <int N1>
MDL_HD int stride(int k) { return k == 0 ? 1 : (k == 1 ? N1 : N1 * N1); }

// Tangential directions of a normal-k face, increasing.
template <int DIM>
MDL_HD void tangents(int k, int* t) {
    int j = 0;
    for (int l = 0; l < DIM; ++l)
        if (l != k) t[j++] = l;
}

// ---------------------------------------------------------------------------
// Volume term.
// ---------------------------------------------------------------------------
template <typename R, int DIM, int P>
MDL_HD void volume_term(const Tables<R>& T, const Phys<R>& ph, int lev, const R* u, R* r) {
    using S = Shape<DIM, P>;
    constexpr int N1 = S::N1, NP = S::NP;
    R G[DIM][NP];
#pragma unroll
    for (int l = 0; l < DIM; ++l) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int a = digit<N1>(q, l);
            const int base = q - a * stride<N1>(l);
            R s = 0;
#pragma unroll
            for (int j = 0; j < N1; ++j) s += T.D1[a][j] * u[base + j * stride<N1>(l)];
            G[l][q] = s * ph.h2[lev][l];
        }
    }
    // H_k = W * sum_l D_kl G_l, stored back into G (per point, all k at once)
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        R wq = ph.Wvol[lev];
#pragma unroll
        for (int l = 0; l < DIM; ++l) wq *= T.w[digit<N1>(q, l)];
        R F[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            R s = 0;
#pragma unroll
            for (int l = 0; l < DIM; ++l) s += ph.D[k][l] * G[l][q];
            F[k] = wq * s;
        }
#pragma unroll
        for (int k = 0; k < DIM; ++k) G[k][q] = F[k];
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int a = digit<N1>(q, k);
            const int base = q - a * stride<N1>(k);
            R s = 0;
#pragma unroll
            for (int i = 0; i < N1; ++i) s += T.D1[i][a] * G[k][base + i * stride<N1>(k)];
            r[q] += ph.h2[lev][k] * s;
        }
    }
}

// ---------------------------------------------------------------------------
// Face evaluation: values and physical gradients of an element's polynomial at
// the points of one of its faces (axis k, side s in {-1,+1}).
// cb < 0: points at the element's own tangential GL nodes.
// cb >= 0: points at the fine GL nodes of the half/quarter (bit t of cb = half
//          along tangent t) of the face -- the element is the coarse side.
// Face point index t = t0 + N1 t1 (t0 along the first tangent).
// ---------------------------------------------------------------------------
template <typename R, int DIM, int P>
MDL_HD void face_eval(const Tables<R>& T, const R* h2, int k, int s, int cb, const R* u,
                      R* val, R grad[DIM][Shape<DIM, P>::NT]) {
    using S = Shape<DIM, P>;
    constexpr int N1 = S::N1, NT = S::NT;
    int tg[2] = {0, 0};
    tangents<DIM>(k, tg);
    const R* bn = (s > 0) ? T.bR : T.bL;
    const R* dn = (s > 0) ? T.dR : T.dL;
    R tr[NT], nd[NT];
#pragma unroll
    for (int m = 0; m < NT; ++m) {
        const int m0 = m % N1, m1 = (DIM == 3) ? m / N1 : 0;
        int base = m0 * stride<N1>(tg[0]);
        if (DIM == 3) base += m1 * stride<N1>(tg[1]);
        R a = 0, b = 0;
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            const R x = u[base + j * stride<N1>(k)];
            a += bn[j] * x;
            b += dn[j] * x;
        }
        tr[m] = a;
        nd[m] = b * h2[k];
    }
    if (cb < 0) {
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            val[t] = tr[t];
            grad[k][t] = nd[t];
        }
#pragma unroll
        for (int ti = 0; ti < DIM - 1; ++ti) {
            const int l = tg[ti];
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int tt = (ti == 0) ? t % N1 : t / N1;
                const int base = t - tt * (ti == 0 ? 1 : N1);
                R acc = 0;
#pragma unroll
                for (int m = 0; m < N1; ++m) acc += T.D1[tt][m] * tr[base + m * (ti == 0 ? 1 : N1)];
                grad[l][t] = acc * h2[l];
            }
        }
    } else {
        const int c0 = cb & 1, c1 = (cb >> 1) & 1;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int t0 = t % N1, t1 = (DIM == 3) ? t / N1 : 0;
            R v = 0, gn = 0, g0 = 0, g1 = 0;
#pragma unroll
            for (int m = 0; m < NT; ++m) {
                const int m0 = m % N1, m1 = (DIM == 3) ? m / N1 : 0;
                R w0 = T.Pi[c0][t0][m0], d0 = T.Pd[c0][t0][m0];
                R w1 = (DIM == 3) ? T.Pi[c1][t1][m1] : R(1);
                R d1 = (DIM == 3) ? T.Pd[c1][t1][m1] : R(0);
                v += w0 * w1 * tr[m];
                gn += w0 * w1 * nd[m];
                g0 += d0 * w1 * tr[m];
                g1 += w0 * d1 * tr[m];
            }
            val[t] = v;
            grad[k][t] = gn;
            grad[tg[0]][t] = g0 * h2[tg[0]];
            if (DIM == 3) grad[tg[1]][t] = g1 * h2[tg[1]];
        }
    }
}

// Adjoint of face_eval for the test functions: r[q] += sum_t cval[t] psi_q(x_t)
// + sum_t sum_l cg[l][t] d_l psi_q(x_t).
template <typename R, int DIM, int P>
MDL_HD void face_adjoint(const Tables<R>& T, const R* h2, int k, int s, int cb, const R* cval,
                         const R cg[DIM][Shape<DIM, P>::NT], R* r) {
    using S = Shape<DIM, P>;
    constexpr int N1 = S::N1, NT = S::NT;
    int tg[2] = {0, 0};
    tangents<DIM>(k, tg);
    const R* bn = (s > 0) ? T.bR : T.bL;
    const R* dn = (s > 0) ? T.dR : T.dL;
    R trc[NT], ndc[NT];
    if (cb < 0) {
#pragma unroll
        for (int m = 0; m < NT; ++m) {
            trc[m] = cval[m];
            ndc[m] = cg[k][m] * h2[k];
        }
#pragma unroll
        for (int ti = 0; ti < DIM - 1; ++ti) {
            const int l = tg[ti];
            const int st = (ti == 0) ? 1 : N1;
#pragma unroll
            for (int m = 0; m < NT; ++m) {
                const int mm = (ti == 0) ? m % N1 : m / N1;
                const int base = m - mm * st;
                R acc = 0;
#pragma unroll
                for (int t = 0; t < N1; ++t) acc += T.D1[t][mm] * cg[l][base + t * st];
                trc[m] += acc * h2[l];
            }
        }
    } else {
        const int c0 = cb & 1, c1 = (cb >> 1) & 1;
#pragma unroll
        for (int m = 0; m < NT; ++m) {
            const int m0 = m % N1, m1 = (DIM == 3) ? m / N1 : 0;
            R a = 0, b = 0;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int t0 = t % N1, t1 = (DIM == 3) ? t / N1 : 0;
                R w0 = T.Pi[c0][t0][m0], d0 = T.Pd[c0][t0][m0];
                R w1 = (DIM == 3) ? T.Pi[c1][t1][m1] : R(1);
                R d1 = (DIM == 3) ? T.Pd[c1][t1][m1] : R(0);
                a += w0 * w1 * cval[t] + d0 * w1 * cg[tg[0]][t] * h2[tg[0]];
                if (DIM == 3) a += w0 * d1 * cg[tg[1]][t] * h2[tg[1]];
                b += w0 * w1 * cg[k][t];
            }
            trc[m] = a;
            ndc[m] = b * h2[k];
        }
    }
#pragma unroll
    for (int m = 0; m < NT; ++m) {
        const int m0 = m % N1, m1 = (DIM == 3) ? m / N1 : 0;
        int base = m0 * stride<N1>(tg[0]);
        if (DIM == 3) base += m1 * stride<N1>(tg[1]);
#pragma unroll
        for (int j = 0; j < N1; ++j) r[base + j * stride<N1>(k)] += bn[j] * trc[m] + dn[j] * ndc[m];
    }
}

// Face point weights W_t = prod_tangential w_{t_l} (h_l / 2) at level `lev` (the finer side).
template <typename R, int DIM, int P>
MDL_HD void face_weights(const Tables<R>& T, const Phys<R>& ph, int lev, int k, R* W) {
    using S = Shape<DIM, P>;
    constexpr int N1 = S::N1, NT = S::NT;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        R w = T.w[t % N1];
        if (DIM == 3) w *= T.w[t / N1];
        W[t] = w * ph.Wface[lev][k];
    }
}

// One (sub)face contribution to the own element's residual.
//   own: values of the own element (level lo), face (k, s), evaluated with cb_own
//   nb : values of the neighbour (level ln), its face (k, -s), evaluated with cb_nb
//   lf : level of the finer side (face points and weights)
template <typename R, int DIM, int P>
MDL_HD void face_term(const Tables<R>& T, const Phys<R>& ph, int k, int s, int lo, int cb_own,
                      const R* own, int ln, int cb_nb, const R* nb, int lf, R* r) {
    using S = Shape<DIM, P>;
    constexpr int NT = S::NT;
    R vo[NT], vn[NT], go[DIM][NT], gn[DIM][NT], W[NT];
    face_eval<R, DIM, P>(T, ph.h2[lo], k, s, cb_own, own, vo, go);
    face_eval<R, DIM, P>(T, ph.h2[ln], k, -s, cb_nb, nb, vn, gn);
    face_weights<R, DIM, P>(T, ph, lf, k, W);
    const R kap = ph.gamma * R(0.5) * (ph.D[k][k] / ph.h[lo][k] + ph.D[k][k] / ph.h[ln][k]);
    const R sg = (s > 0) ? R(1) : R(-1);
    R cval[NT], cg[DIM][NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        R fo = 0, fn = 0;
#pragma unroll
        for (int l = 0; l < DIM; ++l) {
            fo += ph.D[k][l] * go[l][t];
            fn += ph.D[k][l] * gn[l][t];
        }
        const R favg = sg * R(0.5) * (fo + fn);   // {D grad u}.n_own
        const R jump = vo[t] - vn[t];
        cval[t] = W[t] * (kap * jump - favg);
        const R cj = -R(0.5) * W[t] * jump * sg;
#pragma unroll
        for (int l = 0; l < DIM; ++l) cg[l][t] = cj * ph.D[k][l];
    }
    face_adjoint<R, DIM, P>(T, ph.h2[lo], k, s, cb_own, cval, cg, r);
}

// Own-side-only face contribution (neighbour values zero), for the CFL own block.
template <typename R, int DIM, int P>
MDL_HD void face_term_own(const Tables<R>& T, const Phys<R>& ph, int k, int s, int lo, int cb_own,
                          const R* own, int ln, int lf, R* r) {
    R zero[Shape<DIM, P>::NP];
    for (int q = 0; q < Shape<DIM, P>::NP; ++q) zero[q] = 0;
    face_term<R, DIM, P>(T, ph, k, s, lo, cb_own, own, ln, -1, zero, lf, r);
}

// Kelly-type flux jump contribution of one (sub)face (Eq. dg-error-estimate):
//   h_F/(2p) sum_t W_t (W_F [D grad phi . n])^2, h_F = |F|^(1/(d-1)), W_F = |F| / 2^(d-1).
template <typename R, int DIM, int P>
MDL_HD double face_kelly(const Tables<R>& T, const Phys<R>& ph, int k, int s, int lo, int cb_own,
                         const R* own, int ln, int cb_nb, const R* nb, int lf) {
    using S = Shape<DIM, P>;
    constexpr int NT = S::NT;
    R vo[NT], vn[NT], go[DIM][NT], gn[DIM][NT], W[NT];
    face_eval<R, DIM, P>(T, ph.h2[lo], k, s, cb_own, own, vo, go);
    face_eval<R, DIM, P>(T, ph.h2[ln], k, -s, cb_nb, nb, vn, gn);
    face_weights<R, DIM, P>(T, ph, lf, k, W);
    const double WF = (double)ph.Wface[lf][k];
    const double area = WF * (double)(1 << (DIM - 1));
    const double hF = (DIM == 2) ? area : sqrt(area);
    double acc = 0;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        R fo = 0, fn = 0;
#pragma unroll
        for (int l = 0; l < DIM; ++l) {
            fo += ph.D[k][l] * go[l][t];
            fn += ph.D[k][l] * gn[l][t];
        }
        const double j = (double)(fo - fn) * WF;
        acc += (double)W[t] * j * j;
    }
    return hF / (2.0 * P) * acc;
}

// face_kelly without its FP64 factor: sum_t W_t (D grad phi . n jump)^2 in the working
// precision (FP32 on the device, where FP64 runs at a small fraction of the FP32 rate); the
// caller multiplies by kfac = h_F/(2p) W_F^2 and accumulates the faces in FP64.
template <typename R, int DIM, int P>
MDL_HD R face_kelly_sum(const Tables<R>& T, const Phys<R>& ph, int k, int s, int lo, int cb_own, const R* own,
                        int ln, int cb_nb, const R* nb, int lf) {
    using S = Shape<DIM, P>;
    constexpr int NT = S::NT;
    R vo[NT], vn[NT], go[DIM][NT], gn[DIM][NT], W[NT];
    face_eval<R, DIM, P>(T, ph.h2[lo], k, s, cb_own, own, vo, go);
    face_eval<R, DIM, P>(T, ph.h2[ln], k, -s, cb_nb, nb, vn, gn);
    face_weights<R, DIM, P>(T, ph, lf, k, W);
    R acc = 0;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        R fo = 0, fn = 0;
#pragma unroll
        for (int l = 0; l < DIM; ++l) {
            fo += ph.D[k][l] * go[l][t];
            fn += ph.D[k][l] * gn[l][t];
        }
        const R j = fo - fn;
        acc += W[t] * j * j;
    }
    return acc;
}

}  // namespace mdl
