// mdl_mapped.cuh -- the element step on curved (mapped) meshes: thread per element.
//
// The geometric factors of every element (mdl_geometry.h) are stored per GL point: at volume
// node q the symmetric metric G_q and the mass M_q, at face point t the flux vector c, the
// area weight dS and the penalty kappa.  The residual of element e (Eq. monodomain-primal-
// formulation with the flux of Eq. monodomain-numerical-flux, all faces conforming):
//   volume:  r_i += sum_q grad_xi psi_i(q) . G_q grad_xi u(q)
//   face f:  at each point t, with the own trace u_o, the neighbour's trace u_n (its opposite
//            face), flux = c . grad_xi u on each side and jump = u_o - u_n,
//            r_i += dS [ (-(flux_o + flux_n)/2 + kappa jump) psi_i(t) - jump/2 c . grad_xi psi_i(t) ]
// The pointwise update, RV-T term and probe check are those of the box elements with the
// element's own GL mass M_q.
#pragma once

#include "mdl_geofactors.cuh"
#include "mdl_kernels.cuh"

namespace mdl {

template <int DIM, int P>
struct MapShape {
    static constexpr int N1 = P + 1;
    static constexpr int NP = DIM == 2 ? N1 * N1 : N1 * N1 * N1;
    static constexpr int NF = 2 * DIM;
    static constexpr int NPF = DIM == 2 ? N1 : N1 * N1;
    static constexpr int NS = DIM * (DIM + 1) / 2;
    static constexpr int VPN = NS + 1;        // values per volume node: G, M
    static constexpr int FPV = DIM + 2;       // values per face point: c, dS, kappa
};

// Entry (k, l) of the symmetric metric stored as (xx, yy, xy) or (xx, yy, zz, xy, xz, yz).
template <int DIM>
__device__ __forceinline__ int sym_index(int k, int l) {
    if (k == l) return k;
    if (DIM == 2) return 2;
    const int a = k < l ? k : l, b = k < l ? l : k;
    return a == 0 ? (b == 1 ? 3 : 4) : 5;
}

// Tangential axes of a normal-k face, increasing.
template <int DIM>
__device__ __forceinline__ void face_tangents(int k, int* tg) {
    int z = 0;
#pragma unroll
    for (int l = 0; l < DIM; ++l)
        if (l != k) tg[z++] = l;
}

// At the points t of face f = 2k + sd (sd = 1: the +k side), own and neighbour traces (to, tn)
// and the normal fluxes c . grad_xi u of both sides (flo, fln): the normal derivative from
// the 1D derivative values at the face, the tangential ones from the traces by the 1D
// derivative matrix.  The neighbour is seen through its opposite face.
template <typename R, int DIM, int P>
__device__ __forceinline__ void mapped_face_fluxes(const Tables<R>& T, const R* u, const R* un, int k, int sd,
                                                   const R* gf, R* to, R* tn, R* flo, R* fln) {
    using M = MapShape<DIM, P>;
    constexpr int N1 = M::N1, NPF = M::NPF, FPV = M::FPV;
    const R* bs = sd ? T.bR : T.bL;
    const R* ds = sd ? T.dR : T.dL;
    const R* bn = sd ? T.bL : T.bR;
    const R* dn = sd ? T.dL : T.dR;
    int tg[2] = {0, 0};
    face_tangents<DIM>(k, tg);
    R go[NPF], gn[NPF];
#pragma unroll
    for (int t = 0; t < NPF; ++t) {
        const int at0 = t % N1, at1 = t / N1;
        int q0 = at0 * stride<N1>(tg[0]);
        if (DIM == 3) q0 += at1 * stride<N1>(tg[1]);
        R a = 0, b = 0, c = 0, g2 = 0;
#pragma unroll
        for (int m = 0; m < N1; ++m) {
            const int q = q0 + m * stride<N1>(k);
            a += bs[m] * u[q];
            c += ds[m] * u[q];
            b += bn[m] * un[q];
            g2 += dn[m] * un[q];
        }
        to[t] = a;
        go[t] = c;
        tn[t] = b;
        gn[t] = g2;
    }
#pragma unroll
    for (int t = 0; t < NPF; ++t) {
        const int at[2] = {t % N1, t / N1};
        const R* c = gf + t * FPV;
        R fo = c[k] * go[t], fn = c[k] * gn[t];
#pragma unroll
        for (int z = 0; z < DIM - 1; ++z) {
            const int st = z == 0 ? 1 : N1;            // face-point stride of tangent z
            R so = 0, sn = 0;
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                const int t2 = t + (a - at[z]) * st;
                so += T.D1[at[z]][a] * to[t2];
                sn += T.D1[at[z]][a] * tn[t2];
            }
            fo += c[tg[z]] * so;
            fn += c[tg[z]] * sn;
        }
        flo[t] = fo;
        fln[t] = fn;
    }
}

// At a point of face (normal axis k, side sd) of an element with values v whose tangential basis
// rows are L[z][m] and DL[z][m] (d/dxi of the element's own tangential coordinate): the trace and
// cscale * c . grad_xi v.  Used where the point is not one of the element's own face GL points
// (hanging faces: the coarse side at the fine points).
template <typename R, int DIM, int P>
__device__ __forceinline__ void face_point_eval(const Tables<R>& T, const R* v, int k, int sd, const int* tg,
                                                const R (*L)[P + 1], const R (*DL)[P + 1], const R* c, R cscale,
                                                R& tr, R& fl) {
    constexpr int N1 = P + 1;
    const R* bs = sd ? T.bR : T.bL;
    const R* ds = sd ? T.dR : T.dL;
    R t = 0, gn = 0, g0 = 0, g1 = 0;
#pragma unroll
    for (int m = 0; m < N1; ++m)
#pragma unroll
        for (int m0 = 0; m0 < N1; ++m0)
#pragma unroll
            for (int m1 = 0; m1 < (DIM == 3 ? N1 : 1); ++m1) {
                const int node = m * stride<N1>(k) + m0 * stride<N1>(tg[0]) + (DIM == 3 ? m1 * stride<N1>(tg[1]) : 0);
                const R l1 = DIM == 3 ? L[1][m1] : R(1);
                const R val = v[node];
                t += bs[m] * L[0][m0] * l1 * val;
                gn += ds[m] * L[0][m0] * l1 * val;
                g0 += bs[m] * DL[0][m0] * l1 * val;
                if (DIM == 3) g1 += bs[m] * L[0][m0] * DL[1][m1] * val;
            }
    tr = t;
    fl = cscale * (c[k] * gn + c[tg[0]] * g0 + (DIM == 3 ? c[tg[1]] * g1 : R(0)));
}

// r_i += A psi_i + Bc cscale c . grad_xi psi_i at such a point.
template <typename R, int DIM, int P>
__device__ __forceinline__ void face_point_distribute(const Tables<R>& T, int k, int sd, const int* tg,
                                                      const R (*L)[P + 1], const R (*DL)[P + 1], const R* c, R cscale,
                                                      R A, R Bc, R* r) {
    constexpr int N1 = P + 1;
    const R* bs = sd ? T.bR : T.bL;
    const R* ds = sd ? T.dR : T.dL;
    const R Bs = Bc * cscale;
#pragma unroll
    for (int m = 0; m < N1; ++m)
#pragma unroll
        for (int m0 = 0; m0 < N1; ++m0)
#pragma unroll
            for (int m1 = 0; m1 < (DIM == 3 ? N1 : 1); ++m1) {
                const int node = m * stride<N1>(k) + m0 * stride<N1>(tg[0]) + (DIM == 3 ? m1 * stride<N1>(tg[1]) : 0);
                const R l1 = DIM == 3 ? L[1][m1] : R(1);
                const R psi = bs[m] * L[0][m0] * l1;
                const R cg = c[k] * ds[m] * L[0][m0] * l1 + c[tg[0]] * bs[m] * DL[0][m0] * l1 +
                             (DIM == 3 ? c[tg[1]] * bs[m] * L[0][m0] * DL[1][m1] : R(0));
                r[node] += A * psi + Bs * cg;
            }
}

// Tangential basis rows at face point t of a half-face: the coarse side of a hanging face seen at
// the finer side's GL point t, half `bits` (per tangent) of its own face.
template <typename R, int DIM, int P>
__device__ __forceinline__ void half_rows(const Tables<R>& T, int t, int bits, R (*L)[P + 1], R (*DL)[P + 1]) {
    constexpr int N1 = P + 1;
    const int at[2] = {t % N1, t / N1};
#pragma unroll
    for (int z = 0; z < DIM - 1; ++z) {
        const int b = (bits >> z) & 1;
#pragma unroll
        for (int m = 0; m < N1; ++m) {
            L[z][m] = T.Pi[b][at[z]][m];
            DL[z][m] = T.Pd[b][at[z]][m];
        }
    }
}

// The faces of element e with finer neighbours (kind 3 on face f): each subface sb is the
// opposite face of neighbour j = hang[sb], integrated at j's GL points with j's stored factors
// (flux vector c_j along j's outward normal, area weight, penalty).  This element's flux vector
// there is -c_j / 2 (the opposite normal, twice the extent); its trace and gradient come from
// its own values on the half of its face the subface covers.
template <typename R, int DIM, int P>
__device__ __forceinline__ void mapped_hanging_coarse(const DevArrays<R>& d, const Tables<R>& T, int tick, int B,
                                                      int e, int f, const R* u, R* r) {
    using M = MapShape<DIM, P>;
    constexpr int NP = M::NP, NF = M::NF, NPF = M::NPF, FPV = M::FPV, NSUB = 1 << (DIM - 1);
    constexpr int NPS = Shape<DIM, P>::NPS;
    const int k = f >> 1, sd = f & 1;
    int tg[2] = {0, 0};
    face_tangents<DIM>(k, tg);
    const int base = d.nbr[(size_t)e * NF + f];
    for (int sb = 0; sb < NSUB; ++sb) {
        const int j = d.hang[base + sb];
        R uj[NP];
        load_seen<R, NP, NPS>(d, tick, B, j, uj);
        const R* gfj = d.gface + ((size_t)j * NF + (f ^ 1)) * NPF * FPV;
        R tj[NPF], tx[NPF], fj[NPF], fx[NPF];
        mapped_face_fluxes<R, DIM, P>(T, uj, uj, k, sd ^ 1, gfj, tj, tx, fj, fx);
#pragma unroll
        for (int t = 0; t < NPF; ++t) {
            const R* c = gfj + t * FPV;
            R L[2][P + 1], DL[2][P + 1];
            half_rows<R, DIM, P>(T, t, sb, L, DL);
            R tro, flo;
            face_point_eval<R, DIM, P>(T, u, k, sd, tg, L, DL, c, R(-0.5), tro, flo);
            const R fln = -fj[t];
            const R dS = c[DIM], kap = c[DIM + 1];
            const R jump = tro - tj[t];
            const R A = dS * (R(-0.5) * (flo + fln) + kap * jump);
            const R Bc = R(-0.5) * dS * jump;
            face_point_distribute<R, DIM, P>(T, k, sd, tg, L, DL, c, R(-0.5), A, Bc, r);
        }
    }
}

template <typename R, int DIM, int P>
__device__ __forceinline__ void mapped_residual(const DevArrays<R>& d, const Tables<R>& T, int tick, int B, int e,
                                                uint32_t inf, const R* u, R* r) {
    using M = MapShape<DIM, P>;
    constexpr int N1 = M::N1, NP = M::NP, NF = M::NF, NPF = M::NPF, VPN = M::VPN, FPV = M::FPV;
    constexpr int NPS = Shape<DIM, P>::NPS;
#pragma unroll
    for (int q = 0; q < NP; ++q) r[q] = R(0);
    // volume: flux G_q grad u at every node, then r_i = sum_k sum_m D1[m][a_k(i)] flux_k(node m of i's line)
    {
        const R* gv = d.gvol + (size_t)e * NP * VPN;
        R fl[NP][DIM];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            R g[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const int ak = digit<N1>(q, k);
                R s = R(0);
#pragma unroll
                for (int m = 0; m < N1; ++m) s += T.D1[ak][m] * u[q + (m - ak) * stride<N1>(k)];
                g[k] = s;
            }
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                R s = R(0);
#pragma unroll
                for (int l = 0; l < DIM; ++l) s += gv[q * VPN + sym_index<DIM>(k, l)] * g[l];
                fl[q][k] = s;
            }
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            R s = R(0);
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const int ak = digit<N1>(i, k);
#pragma unroll
                for (int m = 0; m < N1; ++m) s += T.D1[m][ak] * fl[i + (m - ak) * stride<N1>(k)][k];
            }
            r[i] = s;
        }
    }
    // faces
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int kind = (inf >> (4 * f)) & 3;
        if (kind == 0) continue;
        const int k = f >> 1, sd = f & 1;
        if (kind == 3) {
            mapped_hanging_coarse<R, DIM, P>(d, T, tick, B, e, f, u, r);
            continue;
        }
        R un[NP];
        load_seen<R, NP, NPS>(d, tick, B, d.nbr[(size_t)e * NF + f], un);
        const R* bs = sd ? T.bR : T.bL;
        const R* ds = sd ? T.dR : T.dL;
        int tg[2] = {0, 0};
        face_tangents<DIM>(k, tg);
        R to[NPF], tn[NPF], flo[NPF], fln[NPF];
        const R* gf = d.gface + ((size_t)e * NF + f) * NPF * FPV;
        mapped_face_fluxes<R, DIM, P>(T, u, un, k, sd, gf, to, tn, flo, fln);
        if (kind == 2) {
            // a coarser neighbour: its trace and flux at this element's points, on the half of
            // its face given by the position bits; its flux vector is half this element's
            const int pos = (inf >> (4 * f + 2)) & 3;
#pragma unroll
            for (int t = 0; t < NPF; ++t) {
                R L[2][P + 1], DL[2][P + 1];
                half_rows<R, DIM, P>(T, t, pos, L, DL);
                face_point_eval<R, DIM, P>(T, un, k, sd ^ 1, tg, L, DL, gf + t * FPV, R(0.5), tn[t], fln[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < NPF; ++t) {
            const int at[2] = {t % N1, t / N1};
            const R* c = gf + t * FPV;
            const R dS = c[DIM], kap = c[DIM + 1];
            const R jump = to[t] - tn[t];
            const R A = dS * (R(-0.5) * (flo[t] + fln[t]) + kap * jump);
            const R Bc = R(-0.5) * dS * jump;
            int q0 = at[0] * stride<N1>(tg[0]);
            if (DIM == 3) q0 += at[1] * stride<N1>(tg[1]);
#pragma unroll
            for (int m = 0; m < N1; ++m) {
                const int i = q0 + m * stride<N1>(k);
                r[i] += A * bs[m] + Bc * c[k] * ds[m];
#pragma unroll
                for (int z = 0; z < DIM - 1; ++z) {
                    const R w = Bc * c[tg[z]] * bs[m];
#pragma unroll
                    for (int a = 0; a < N1; ++a) r[i + (a - at[z]) * stride<N1>(tg[z])] += w * T.D1[at[z]][a];
                }
            }
        }
    }
}

// One element step of Alg. 1 on a mapped mesh (see tick_elem for the box elements).
template <typename R, int DIM, int P>
__device__ __forceinline__ void tick_elem_mapped(const TickArgs<R>& a, const Tables<R>& T, const Phys<R>& ph,
                                                 int tick, int e) {
    using M = MapShape<DIM, P>;
    constexpr int NP = M::NP, VPN = M::VPN;
    constexpr int NPS = Shape<DIM, P>::NPS;
    const DevArrays<R>& d = a.d;
    const uint8_t lvb = d.lvl[e];
    const uint32_t inf = d.info[e];
    const int b = lvb & 7, par = (lvb >> 3) & 1;
    const int ke = tick >> (a.B - b);
    const int cur = par ^ (ke & 1);
    const R* Vc = (cur ? d.V1 : d.V0) + (size_t)e * NPS;
    R* Vd = (cur ? d.V0 : d.V1) + (size_t)e * NPS;
    R* vp = d.v + (size_t)e * NPS;
    R u[NP], w[NP], r[NP], Ia[NP], ga[NP];
    ld_dofs<R, NP, NPS>(Vc, u);
    ld_dofs<R, NP, NPS>(vp, w);
    mapped_residual<R, DIM, P>(d, T, tick, a.B, e, inf, u, r);
    double acc0 = 0.0;
    if (ke != 0) {
        ld_dofs<R, NP, NPS>(d.Ia + (size_t)e * NPS, Ia);
        ld_dofs<R, NP, NPS>(d.ga + (size_t)e * NPS, ga);
        acc0 = d.acc[e];
    }
    bool stim = false;
    for (int s = 0; s < a.stim.n; ++s) stim = stim || d.smask[s][e] != 0u;
    const double dte_d = a.dte[b];
    const R dte = a.dteR[b];
    const R* gv = d.gvol + (size_t)e * NP * VPN;
    R un[NP], wn[NP];
    R term = R(0), vmax = R(0);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        R so = R(0), sm = R(0);
        if (stim) dof_stim<R>(a, e, tick, dte_d, q, so, sm);
        const R Mq = gv[q * VPN + VPN - 1];
        term += dof_update<R>(ph, Mq, R(1) / Mq, ke, dte, so, sm, u[q], w[q], r[q], Ia[q], ga[q], un[q], wn[q]);
        const R av = un[q] < R(0) ? -un[q] : un[q];
        vmax = av > vmax ? av : vmax;
    }
    if (ke == 0 && b > 0) {
        st_dofs<R, NP, NPS>(d.Ia + (size_t)e * NPS, Ia);
        st_dofs<R, NP, NPS>(d.ga + (size_t)e * NPS, ga);
    }
    st_dofs<R, NP, NPS>(Vd, un);
    st_dofs<R, NP, NPS>(vp, wn);
    d.acc[e] = acc0 + dte_d * (double)term;
    if ((inf & INFO_PENDING) && vmax >= ph.lat_gate) {
        const int lev = (inf >> 24) & 15;
        lat_check<R, DIM, P>(d, T, ph, e, inf, lev, u, un, tick_time(a, tick), dte_d);
    }
}

// Kelly-type spatial indicator (Eq. dg-error-estimate) on the mapped mesh, on the barrier-start
// values: per interior face, with the flux jump J_t = (c . grad_xi u)_own - (c . grad_xi u)_nb,
// the face area |F| = sum_t dS_t, h_F = |F|^(1/(d-1)) and the face map's Jacobian at the point
// W_F(t) = dS_t / (reference GL weight of t): h_F / (2p) sum_t dS_t (W_F(t) J_t)^2.  Face-point
// sums in the working precision, faces accumulated in FP64.
template <typename R, int DIM, int P>
__global__ void __launch_bounds__(128) k_eta_s_mapped(const DevArrays<R> d, const Tables<R> T) {
    pdl_enter();
    using M = MapShape<DIM, P>;
    constexpr int N1 = M::N1, NP = M::NP, NF = M::NF, NPF = M::NPF, FPV = M::FPV;
    constexpr int NPS = Shape<DIM, P>::NPS;
    if (d.meta->err) return;
    const int64_t ne = d.meta->ne;
    for (int64_t e = gtid(); e < ne; e += gstride()) {
        const uint32_t inf = d.info[e];
        const int par = (d.lvl[e] >> 3) & 1;
        R u[NP];
        ld_dofs<R, NP, NPS>((par ? d.V1 : d.V0) + (size_t)e * NPS, u);
        double acc = 0.0;
        // one (sub)face: h_F / (2p) sum_t dS_t (W_F(t) J_t)^2 from its points' area weights and jumps
        auto face_sum = [&](const R* dS, const R* jmp) {
            R area = R(0), sum = R(0);
#pragma unroll
            for (int t = 0; t < NPF; ++t) {
                const R wref = T.w[t % N1] * (DIM == 3 ? T.w[t / N1] : R(1));
                const R x = dS[t] / wref * jmp[t];
                area += dS[t];
                sum += dS[t] * x * x;
            }
            const double hF = DIM == 3 ? sqrt((double)area) : (double)area;
            acc += hF / (2.0 * P) * (double)sum;
        };
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const int kind = (inf >> (4 * f)) & 3;
            if (kind == 0) continue;
            const int k = f >> 1, sd = f & 1;
            int tg[2] = {0, 0};
            face_tangents<DIM>(k, tg);
            const int nb = d.nbr[(size_t)e * NF + f];
            if (kind == 3) {
                // the finer neighbours' subfaces, at their points with their factors
                for (int sb = 0; sb < (1 << (DIM - 1)); ++sb) {
                    const int j = d.hang[nb + sb];
                    R uj[NP];
                    ld_dofs<R, NP, NPS>((((d.lvl[j] >> 3) & 1) ? d.V1 : d.V0) + (size_t)j * NPS, uj);
                    const R* gfj = d.gface + ((size_t)j * NF + (f ^ 1)) * NPF * FPV;
                    R tj[NPF], tx[NPF], fj[NPF], fx[NPF], dS[NPF], jmp[NPF];
                    mapped_face_fluxes<R, DIM, P>(T, uj, uj, k, sd ^ 1, gfj, tj, tx, fj, fx);
#pragma unroll
                    for (int t = 0; t < NPF; ++t) {
                        R L[2][P + 1], DL[2][P + 1];
                        half_rows<R, DIM, P>(T, t, sb, L, DL);
                        R tro, flo;
                        face_point_eval<R, DIM, P>(T, u, k, sd, tg, L, DL, gfj + t * FPV, R(-0.5), tro, flo);
                        jmp[t] = flo + fj[t];
                        dS[t] = gfj[t * FPV + DIM];
                    }
                    face_sum(dS, jmp);
                }
                continue;
            }
            R un[NP];
            ld_dofs<R, NP, NPS>((((d.lvl[nb] >> 3) & 1) ? d.V1 : d.V0) + (size_t)nb * NPS, un);
            const R* gf = d.gface + ((size_t)e * NF + f) * NPF * FPV;
            R to[NPF], tn[NPF], flo[NPF], fln[NPF], dS[NPF], jmp[NPF];
            mapped_face_fluxes<R, DIM, P>(T, u, un, k, sd, gf, to, tn, flo, fln);
            if (kind == 2) {
                const int pos = (inf >> (4 * f + 2)) & 3;
#pragma unroll
                for (int t = 0; t < NPF; ++t) {
                    R L[2][P + 1], DL[2][P + 1];
                    half_rows<R, DIM, P>(T, t, pos, L, DL);
                    face_point_eval<R, DIM, P>(T, un, k, sd ^ 1, tg, L, DL, gf + t * FPV, R(0.5), tn[t], fln[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < NPF; ++t) {
                jmp[t] = flo[t] - fln[t];
                dS[t] = gf[t * FPV + DIM];
            }
            face_sum(dS, jmp);
        }
        d.eta_s[e] = sqrt(acc);
    }
}

// Inputs of the device factor pass: the map and diffusion, FP64 tables, GL nodes, level-0
// extents, stimulus boxes (slack applied), the barrier step and the LTS budget.
struct MapArgs {
    GeoArgs g;
    double xg[3];
    double h0[3];
    int nstim;
    double slo[MDL_MAX_STIM][3], shi[MDL_MAX_STIM][3];
    double dt;
    int B, lts;
};

// Smallest b >= 0 with dt 2^-b <= bound (15 if none below 60; Eq. num-substeps, exact).
__device__ __forceinline__ int b_from_bound_dev(double dt, double bound) {
    for (int b = 0; b <= 60; ++b)
        if (ldexp(dt, -b) <= bound) return b > 15 ? 15 : b;
    return 15;
}

// Factors of the current mesh after an adaptation, part 1.  An element kept by the adaptation
// (pkind 0) with the face kinds it had takes its old factors, GL masses, signature (face kinds
// in bits 0-11, level in bits 12-15, b^CFL in bits 16-19) and stimulus masks (source psrc in the
// old set); a warp walks 32 consecutive elements and copies each kept element's factor rows with
// its lanes (coalesced).  Every other element is appended to `todo` (count m->nfac, zeroed by
// the scan that commits the new mesh) for k_mapped_factors.  Without an old set (o* null)
// every element is appended.
template <typename R, int DIM, int P>
__global__ void __launch_bounds__(256) k_mapped_keep(
        const uint32_t* info, const int nstim, R* gvol, R* gface, double* mass, uint32_t* fsig, uint32_t* f0,
        uint32_t* f1, uint32_t* f2, uint32_t* f3, uint8_t* bcfl, uint32_t* sm0, uint32_t* sm1, uint32_t* sm2,
        uint32_t* sm3, const R* ogvol, const R* ogface, const double* omass, const uint32_t* ofsig,
        const uint32_t* of0, const uint32_t* of1, const uint32_t* of2, const uint32_t* of3, const int8_t* pkind,
        const int32_t* psrc, int32_t* todo, DevMeta* m) {
    pdl_enter();
    using M = MapShape<DIM, P>;
    constexpr int NP = M::NP, NF = M::NF;
    constexpr int NV = NP * M::VPN, NFV = NF * M::NPF * M::FPV;
    if (m->err) return;
    uint32_t* smask[4] = {sm0, sm1, sm2, sm3};
    uint32_t* fsm[4] = {f0, f1, f2, f3};
    const uint32_t* ofsm[4] = {of0, of1, of2, of3};
    const int64_t ne = m->ne;
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = gstride() >> 5;
    for (int64_t base = (gtid() >> 5) * 32; base < ne; base += nwarp * 32) {
        const int64_t e = base + lane;
        bool keep = false;
        int64_t o = 0;
        if (e < ne && ofsig) {
            const uint32_t inf = info[e];
            uint32_t kbits = 0;
            for (int f = 0; f < NF; ++f) kbits |= ((inf >> (4 * f)) & 3u) << (2 * f);
            if (pkind[e] == 0) {
                o = psrc[e];
                const uint32_t sg = ofsig[o];
                keep = (sg & 0xfffu) == kbits;
                if (keep) {
                    fsig[e] = sg;
                    bcfl[e] = (uint8_t)((sg >> 16) & 15u);
                    for (int s = 0; s < nstim; ++s) smask[s][e] = fsm[s][e] = ofsm[s][o];
                }
            }
        }
        const unsigned need = __ballot_sync(0xffffffffu, e < ne && !keep);
        if (need) {
            int slot = 0;
            if (lane == 0) slot = (int)atomicAdd(&m->nfac, (unsigned)__popc(need));
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if ((need >> lane) & 1u) todo[slot + __popc(need & ((1u << lane) - 1u))] = (int32_t)e;
        }
        for (unsigned kept = __ballot_sync(0xffffffffu, keep); kept; kept &= kept - 1u) {
            const int l = __ffs(kept) - 1;
            const int64_t ek = base + l, ok = __shfl_sync(0xffffffffu, o, l);
            for (int i = lane; i < NV; i += 32) gvol[(size_t)ek * NV + i] = ogvol[(size_t)ok * NV + i];
            for (int i = lane; i < NFV; i += 32) gface[(size_t)ek * NFV + i] = ogface[(size_t)ok * NFV + i];
            for (int i = lane; i < NP; i += 32) mass[(size_t)ek * NP + i] = omass[(size_t)ok * NP + i];
        }
    }
}

// One element's factors computed by a whole warp: the arithmetic of geo_element, with the lanes
// over the element's GL points (map, metric, face factors; chunks of 32 points) and over the
// entries of its own block B (registers; every entry summed over the points in geo_element's
// order).  FP64 issues at a small fraction of the FP32 rate on this GPU, so one element's
// instructions are spread over 32 lanes rather than run by one.
template <int DIM, int P>
struct GeoWarp {
    static constexpr int N1 = P + 1;
    static constexpr int NP = DIM == 2 ? N1 * N1 : N1 * N1 * N1;
    static constexpr int NF = 2 * DIM, NPF = DIM == 2 ? N1 : N1 * N1, NSUB = 1 << (DIM - 1);
    static constexpr int NS = DIM * (DIM + 1) / 2, VPN = NS + 1, FPV = DIM + 2;
    static constexpr int CH = 32;                   // points per chunk (one per lane)
    static constexpr int PS = 2 * NP + 2;           // doubles per point: psi, c.grad psi, dS, kappa (face);
                                                    // the metric K (volume node)
    static constexpr int NE = (NP * NP + 31) / 32;  // block entries per lane
    static_assert(PS >= DIM * DIM && CH * PS >= NP * NP, "point record too small");
};

// Returns the Gershgorin bound (every lane); writes the element's volume factors and GL masses
// (gvol, gface, mass: the element's rows) and returns its stimulus masks in sk (every lane).
// spt: CH * PS doubles and sm: NP doubles of shared memory owned by the warp.
template <typename R, int DIM, int P>
__device__ double geo_element_warp(const GeoArgs& g, const Tables<double>& T, const double* xg, const double* h0,
                                   int lev, const int* cc, const int* kinds, int nstim, const double (*slo)[3],
                                   const double (*shi)[3], double* spt, double* sm, R* gvol, R* gface, double* mass,
                                   uint32_t* sk) {
    using W = GeoWarp<DIM, P>;
    constexpr int N1 = W::N1, NP = W::NP, NF = W::NF, NPF = W::NPF, NS = W::NS, VPN = W::VPN, FPV = W::FPV;
    constexpr int CH = W::CH, PS = W::PS, NE = W::NE;
    const int lane = threadIdx.x & 31;
    double h[3] = {1.0, 1.0, 1.0}, Xc[3] = {0.0, 0.0, 0.0}, s2h[3] = {2.0, 2.0, 2.0};
    const double sc = 1.0 / (double)(1 << lev);
    for (int k = 0; k < DIM; ++k) {
        h[k] = h0[k] * sc;
        Xc[k] = cc[k] * h[k];
        s2h[k] = 2.0 / h[k];
    }
    // points: the NP volume nodes, then per face with a neighbour its GL points (kind 3: the
    // finer neighbours' points, subface outer)
    int off[NF + 1];
    off[0] = NP;
    for (int f = 0; f < NF; ++f) off[f + 1] = off[f] + (kinds[f] ? NPF * (kinds[f] == 3 ? W::NSUB : 1) : 0);
    const int npt = off[NF];
    for (int f = 0; f < NF; ++f)
        if (kinds[f] == 0 || kinds[f] == 3)
            for (int i = lane; i < NPF * FPV; i += 32) gface[f * NPF * FPV + i] = (R)0;
    uint32_t mk[MDL_MAX_STIM] = {0u, 0u, 0u, 0u};
    double bacc[NE];
#pragma unroll
    for (int u = 0; u < NE; ++u) bacc[u] = 0.0;
    for (int c0 = 0; c0 < npt; c0 += CH) {
        const int p = c0 + lane;
        double* rec = spt + lane * PS;
        if (p < NP) {
            const int q = p;
            double X[3] = {0.0, 0.0, 0.0}, x[3], J[3][3], Ji[3][3], D[3][3];
            double Wq = 1.0;
            for (int k = 0; k < DIM; ++k) {
                const int a = digit<N1>(q, k);
                X[k] = Xc[k] + (xg[a] + 1.0) * 0.5 * h[k];
                Wq *= T.w[a] * h[k] * 0.5;
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
                    K[i][j] = Wq * fabs(det) * s2h[i] * s * s2h[j];
                    rec[i * DIM + j] = K[i][j];
                }
            R* gv = gvol + q * VPN;
            if (DIM == 2) {
                gv[0] = (R)K[0][0]; gv[1] = (R)K[1][1]; gv[2] = (R)K[0][1];
            } else {
                gv[0] = (R)K[0][0]; gv[1] = (R)K[1][1]; gv[2] = (R)K[2][2];
                gv[3] = (R)K[0][1]; gv[4] = (R)K[0][2]; gv[5] = (R)K[1][2];
            }
            const double mq = Wq * fabs(det);
            mass[q] = mq;
            gv[NS] = (R)mq;
            sm[q] = mq;
            for (int s = 0; s < nstim; ++s) {
                bool in = true;
                for (int k = 0; k < DIM; ++k) in = in && x[k] >= slo[s][k] && x[k] <= shi[s][k];
                if (in) mk[s] |= 1u << q;
            }
        } else if (p < npt) {
            int f = 0;
            while (off[f + 1] <= p) ++f;
            const int kind = kinds[f], r = p - off[f], sb = r / NPF, t = r - sb * NPF;
            const int k = f >> 1, sd = f & 1;
            const double sgn = sd ? 1.0 : -1.0;
            int tg[2] = {0, 0}, nt = 0;
            for (int l = 0; l < DIM; ++l)
                if (l != k) tg[nt++] = l;
            const double* bs = sd ? T.bR : T.bL;
            const double* ds = sd ? T.dR : T.dL;
            const double pen = kind == 2 ? 0.75 : (kind == 3 ? 1.5 : 1.0);   // (1 + h_own / h_nb) / 2
            const int at[2] = {t % N1, t / N1};
            double X[3] = {0.0, 0.0, 0.0};
            double Wt = 1.0;
            double xi_t[2] = {0.0, 0.0};
            X[k] = Xc[k] + (sd ? h[k] : 0.0);
            for (int z = 0; z < nt; ++z) {
                const int l = tg[z];
                if (kind == 3) {
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
            geo_face_point(g, X, h, k, sgn, c, &adet, &ln, &nDn);
            const double dS = Wt * adet * ln;
            const double kap = g.gamma * nDn * ln / h[k] * pen;
            if (sb == 0 && kind != 3) {
                R* gf = gface + (f * NPF + t) * FPV;
                for (int i = 0; i < DIM; ++i) gf[i] = (R)c[i];
                gf[DIM] = (R)dS;
                gf[DIM + 1] = (R)kap;
            }
            double lt[2][3], dlt[2][3];
            for (int z = 0; z < nt; ++z) geo_lagrange<N1>(xg, xi_t[z], lt[z], dlt[z]);
            for (int i = 0; i < NP; ++i) {
                const int ak = digit<N1>(i, k);
                double tv = 1.0;
                for (int z = 0; z < nt; ++z) tv *= lt[z][digit<N1>(i, tg[z])];
                double cgi = c[k] * ds[ak] * tv;
                for (int z = 0; z < nt; ++z) {
                    double dz = bs[ak] * dlt[z][digit<N1>(i, tg[z])];
                    for (int z2 = 0; z2 < nt; ++z2)
                        if (z2 != z) dz *= lt[z2][digit<N1>(i, tg[z2])];
                    cgi += c[tg[z]] * dz;
                }
                rec[i] = bs[ak] * tv;
                rec[NP + i] = cgi;
            }
            rec[2 * NP] = dS;
            rec[2 * NP + 1] = kap;
        }
        __syncwarp();
        // block entries (i, j) = (ent / NP, ent % NP), ent = lane + 32 u, summed over the chunk's points
        const int pe = min(CH, npt - c0);
        for (int pp = 0; pp < pe; ++pp) {
            const double* d = spt + pp * PS;
            if (c0 + pp < NP) {
                // volume node q: B_ij += g_i^T K g_j, g_i = grad psi_i at q (nonzero when i and q
                // differ in at most one digit k: D1[q_k][i_k] there)
                const int q = c0 + pp;
#pragma unroll
                for (int u = 0; u < NE; ++u) {
                    const int ent = lane + 32 * u;
                    if (ent >= NP * NP) continue;
                    const int i = ent / NP, j = ent - (ent / NP) * NP;
                    int di = 0, ki = 0, dj = 0, kj = 0;
                    for (int k = 0; k < DIM; ++k) {
                        if (digit<N1>(i, k) != digit<N1>(q, k)) { ++di; ki = k; }
                        if (digit<N1>(j, k) != digit<N1>(q, k)) { ++dj; kj = k; }
                    }
                    if (di > 1 || dj > 1) continue;
                    double s = bacc[u];
                    for (int k = 0; k < DIM; ++k) {
                        if (di == 1 && k != ki) continue;
                        const double gik = T.D1[digit<N1>(q, k)][digit<N1>(i, k)];
                        for (int l = 0; l < DIM; ++l) {
                            if (dj == 1 && l != kj) continue;
                            s += gik * d[k * DIM + l] * T.D1[digit<N1>(q, l)][digit<N1>(j, l)];
                        }
                    }
                    bacc[u] = s;
                }
            } else {
                const double dS = d[2 * NP], kap = d[2 * NP + 1];
#pragma unroll
                for (int u = 0; u < NE; ++u) {
                    const int ent = lane + 32 * u;
                    if (ent >= NP * NP) continue;
                    const int i = ent / NP, j = ent - (ent / NP) * NP;
                    const double pi = d[i], ci = d[NP + i];
                    if (pi == 0.0 && ci == 0.0) continue;
                    bacc[u] += dS * (-0.5 * d[NP + j] * pi - 0.5 * ci * d[j] + kap * pi * d[j]);
                }
            }
        }
        __syncwarp();
    }
    // Gershgorin: max_i sum_j |B_ij| / M_i
#pragma unroll
    for (int u = 0; u < NE; ++u) {
        const int ent = lane + 32 * u;
        if (ent < NP * NP) spt[ent] = fabs(bacc[u]);
    }
    __syncwarp();
    double mx = 0.0;
    if (lane < NP) {
        double row = 0.0;
        for (int j = 0; j < NP; ++j) row += spt[lane * NP + j];
        mx = row / sm[lane];
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    for (int s = 0; s < nstim; ++s) sk[s] = __reduce_or_sync(0xffffffffu, mk[s]);
    __syncwarp();
    return 1.0 / mx;
}

// Part 2: the factors of the listed elements (todo[0 .. m->nfac)), one warp per element
// (geo_element_warp), with their b^CFL, signature and stimulus masks.  List entry j goes to
// warp j mod (number of warps), the warps numbered block-fastest, so that a run of neighbouring
// elements (a refined patch) spreads over every SM.
template <typename R, int DIM, int P>
__global__ void __launch_bounds__(64) k_mapped_factors(
        const int4* coord, const uint32_t* info, const MapArgs a, const Tables<double> Td, R* gvol, R* gface,
        double* mass, uint32_t* fsig, uint32_t* f0, uint32_t* f1, uint32_t* f2, uint32_t* f3, uint8_t* bcfl,
        uint32_t* sm0, uint32_t* sm1, uint32_t* sm2, uint32_t* sm3, const int32_t* todo, DevMeta* m) {
    pdl_enter();
    using W = GeoWarp<DIM, P>;
    constexpr int NP = W::NP, NF = W::NF;
    constexpr int NV = NP * W::VPN, NFV = NF * W::NPF * W::FPV;
    __shared__ double s_pt[2][W::CH * W::PS];
    __shared__ double s_m[2][NP];
    if (m->err) return;
    uint32_t* smask[4] = {sm0, sm1, sm2, sm3};
    uint32_t* fsm[4] = {f0, f1, f2, f3};
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = m->nfac;
    if (blockIdx.x == 0 && threadIdx.x == 0) m->fac_updates += n;
    for (int64_t j = blockIdx.x + (int64_t)gridDim.x * wib; j < n; j += 2 * (int64_t)gridDim.x) {
        const int64_t e = todo[j];
        const int4 c4 = coord[e];
        const uint32_t inf = info[e];
        uint32_t kbits = 0;
        int kinds[6] = {0, 0, 0, 0, 0, 0};
        for (int f = 0; f < NF; ++f) {
            kinds[f] = (inf >> (4 * f)) & 3;
            kbits |= (uint32_t)kinds[f] << (2 * f);
        }
        const int cc[3] = {c4.x, c4.y, c4.z};
        uint32_t sk[MDL_MAX_STIM] = {0u, 0u, 0u, 0u};
        const double cfl = geo_element_warp<R, DIM, P>(a.g, Td, a.xg, a.h0, c4.w, cc, kinds, a.nstim, a.slo, a.shi,
                                                       s_pt[wib], s_m[wib], gvol + (size_t)e * NV,
                                                       gface + (size_t)e * NFV, mass + (size_t)e * NP, sk);
        if (lane == 0) {
            const int b = a.lts ? b_from_bound_dev(a.dt, cfl) : 0;
            bcfl[e] = (uint8_t)b;
            fsig[e] = kbits | ((uint32_t)c4.w << 12) | ((uint32_t)b << 16);
            for (int s = 0; s < a.nstim; ++s) smask[s][e] = fsm[s][e] = sk[s];
        }
    }
}

template <typename R, int DIM, int P>
__global__ void __launch_bounds__(128) k_tick_mapped(const TickArgs<R> a, const Tables<R> T, const Phys<R> ph) {
    const int n_act = a.d.meta->nact[a.tick];
    const bool bad = a.d.meta->err != 0;
    pdl_enter();
    if (bad) return;
    for (int idx = (int)gtid(); idx < n_act; idx += (int)gstride()) tick_elem_mapped<R, DIM, P>(a, T, ph, a.tick, a.d.order[idx]);
}

}  // namespace mdl
