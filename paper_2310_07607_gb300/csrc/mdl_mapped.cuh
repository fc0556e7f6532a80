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

// Every element's geometric factors, GL masses, signature (face kinds in bits 0-11, b^CFL in
// bits 16-19) and stimulus masks on the current mesh, and the shared b^CFL and mask tables.  An
// element kept by the adaptation (pkind 0) with the face kinds it had takes its old values
// (source psrc in the old set); the others are computed in FP64 (geo_element, shared with the
// host).  Without an old set (o* null) every element is computed.
template <typename R, int DIM, int P>
__global__ void __launch_bounds__(64) k_mapped_factors(
        const int4* coord, const uint32_t* info, const MapArgs a, const Tables<double> Td, R* gvol, R* gface,
        double* mass, uint32_t* fsig, uint32_t* f0, uint32_t* f1, uint32_t* f2, uint32_t* f3, uint8_t* bcfl,
        uint32_t* sm0, uint32_t* sm1, uint32_t* sm2, uint32_t* sm3, const R* ogvol, const R* ogface,
        const double* omass, const uint32_t* ofsig, const uint32_t* of0, const uint32_t* of1, const uint32_t* of2,
        const uint32_t* of3, const int8_t* pkind, const int32_t* psrc, DevMeta* m) {
    pdl_enter();
    using M = MapShape<DIM, P>;
    constexpr int NP = M::NP, NF = M::NF, NPF = M::NPF, VPN = M::VPN, FPV = M::FPV;
    constexpr int NV = NP * VPN, NFV = NF * NPF * FPV;
    if (m->err) return;
    uint32_t* smask[4] = {sm0, sm1, sm2, sm3};
    uint32_t* fsm[4] = {f0, f1, f2, f3};
    const uint32_t* ofsm[4] = {of0, of1, of2, of3};
    const int64_t ne = m->ne;
    for (int64_t e = gtid(); e < ne; e += gstride()) {
        const int4 c4 = coord[e];
        const uint32_t inf = info[e];
        uint32_t kbits = 0;
        int kinds[6] = {0, 0, 0, 0, 0, 0};
        for (int f = 0; f < NF; ++f) {
            kinds[f] = (inf >> (4 * f)) & 3;
            kbits |= (uint32_t)kinds[f] << (2 * f);
        }
        if (ofsig && pkind[e] == 0 && (ofsig[psrc[e]] & 0xfffu) == kbits) {
            const int64_t o = psrc[e];
            for (int i = 0; i < NV; ++i) gvol[(size_t)e * NV + i] = ogvol[(size_t)o * NV + i];
            for (int i = 0; i < NFV; ++i) gface[(size_t)e * NFV + i] = ogface[(size_t)o * NFV + i];
            for (int q = 0; q < NP; ++q) mass[(size_t)e * NP + q] = omass[(size_t)o * NP + q];
            const uint32_t sg = ofsig[o];
            fsig[e] = sg;
            bcfl[e] = (uint8_t)((sg >> 16) & 15u);
            for (int s = 0; s < a.nstim; ++s) smask[s][e] = fsm[s][e] = ofsm[s][o];
            continue;
        }
        const int cc[3] = {c4.x, c4.y, c4.z};
        double gv[NV], gf[NFV], ms[NP], Bs[NP * NP];
        uint32_t sk[MDL_MAX_STIM] = {0u, 0u, 0u, 0u};
        const double cfl = geo_element<DIM, P>(a.g, Td, a.xg, a.h0, c4.w, cc, kinds, a.nstim, a.slo, a.shi, gv, gf,
                                               ms, sk, Bs);
        for (int i = 0; i < NV; ++i) gvol[(size_t)e * NV + i] = (R)gv[i];
        for (int i = 0; i < NFV; ++i) gface[(size_t)e * NFV + i] = (R)gf[i];
        for (int q = 0; q < NP; ++q) mass[(size_t)e * NP + q] = ms[q];
        const int b = a.lts ? b_from_bound_dev(a.dt, cfl) : 0;
        bcfl[e] = (uint8_t)b;
        fsig[e] = kbits | ((uint32_t)c4.w << 12) | ((uint32_t)b << 16);
        for (int s = 0; s < a.nstim; ++s) smask[s][e] = fsm[s][e] = sk[s];
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
