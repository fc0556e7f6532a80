// mdl_tables.cpp -- basis tables, physics constants and Gershgorin CFL classes (host, FP64).
#include "mdl_tables.h"

#include <math.h>

#include <cmath>
#include <string.h>

#include <vector>

namespace mdl {

void gl_nodes(int p, double* x, double* w) {
    if (p == 1) {
        const double a = 1.0 / sqrt(3.0);
        x[0] = -a; x[1] = a;
        w[0] = 1.0; w[1] = 1.0;
    } else {
        const double a = sqrt(0.6);
        x[0] = -a; x[1] = 0.0; x[2] = a;
        w[0] = 5.0 / 9.0; w[1] = 8.0 / 9.0; w[2] = 5.0 / 9.0;
    }
}

namespace {

double lag(const double* x, int n, int j, double t) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != j) v *= (t - x[m]) / (x[j] - x[m]);
    return v;
}

double dlag(const double* x, int n, int j, double t) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
        if (k == j) continue;
        double term = 1.0 / (x[j] - x[k]);
        for (int m = 0; m < n; ++m)
            if (m != j && m != k) term *= (t - x[m]) / (x[j] - x[m]);
        s += term;
    }
    return s;
}

}  // namespace

void make_tables(int p, Tables<double>* T) {
    memset(T, 0, sizeof(*T));
    const int n = p + 1;
    double x[3], w[3];
    gl_nodes(p, x, w);
    for (int i = 0; i < n; ++i) {
        T->w[i] = w[i];
        T->bL[i] = lag(x, n, i, -1.0);
        T->bR[i] = lag(x, n, i, 1.0);
        T->dL[i] = dlag(x, n, i, -1.0);
        T->dR[i] = dlag(x, n, i, 1.0);
        for (int j = 0; j < n; ++j) T->D1[i][j] = dlag(x, n, j, x[i]);
    }
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < n; ++i) {
            const double t = (x[i] + 2.0 * c - 1.0) * 0.5;
            for (int m = 0; m < n; ++m) {
                T->Pi[c][i][m] = lag(x, n, m, t);
                T->Pd[c][i][m] = dlag(x, n, m, t);
            }
        }
    // probe lattice: root node a at level l lies in the level-l cell floor((x_a+1)/2 2^l)
    // of its root; rho = its reference coordinate inside that cell.
    for (int l = 0; l < 8; ++l)
        for (int a = 0; a < n; ++a) {
            const double s = (x[a] + 1.0) * 0.5 * (double)(1 << l);
            const int cell = (int)floor(s);
            T->pfl[l][a] = cell;
            const double rho = (s - cell) * 2.0 - 1.0;
            for (int j = 0; j < n; ++j) T->pphi[l][a][j] = lag(x, n, j, rho);
        }
}

void make_phys(const mdl_problem& pb, const Tables<double>& T, Phys<double>* ph) {
    memset(ph, 0, sizeof(*ph));
    const int d = pb.dim;
    double f[3] = {pb.fibre[0], pb.fibre[1], d == 3 ? pb.fibre[2] : 0.0};
    double nf = 0.0;
    for (int k = 0; k < d; ++k) nf += f[k] * f[k];
    nf = sqrt(nf);
    if (nf > 0) {
        for (int k = 0; k < d; ++k) f[k] /= nf;
    } else {
        f[0] = 1.0; f[1] = 0.0; f[2] = 0.0;
    }
    const double s = 1.0 / (pb.chi * pb.cm);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            ph->D[i][j] = (i < d && j < d)
                              ? s * ((i == j ? pb.sigma_t : 0.0) + (pb.sigma_l - pb.sigma_t) * f[i] * f[j])
                              : 0.0;
    ph->gamma = pb.gamma;
    for (int l = 0; l < 8; ++l) {
        double vol = 1.0;
        for (int k = 0; k < 3; ++k) {
            const double h = (k < d) ? pb.extent[k] / ((double)pb.base[k] * (double)(1 << l)) : 1.0;
            ph->h[l][k] = h;
            ph->h2[l][k] = 2.0 / h;
            if (k < d) vol *= h * 0.5;
        }
        ph->Wvol[l] = vol;
        for (int k = 0; k < 3; ++k) {
            double wf = 1.0;
            for (int m = 0; m < d; ++m)
                if (m != k) wf *= ph->h[l][m] * 0.5;
            ph->Wface[l][k] = wf;
            const double area = wf * (double)(1 << (d - 1));
            const double hF = (d == 2) ? area : std::sqrt(area);
            ph->kfac[l][k] = hF / (2.0 * pb.order) * wf * wf;
        }
    }
    const int n1 = pb.order + 1;
    for (int l = 0; l < 8; ++l)
        for (int q = 0; q < 27; ++q) {
            double m = ph->Wvol[l];
            int r = q;
            for (int k = 0; k < d; ++k, r /= n1) m *= T.w[r % n1];
            ph->Minv[l][q] = 1.0 / m;
        }
    ph->ionic = pb.ionic_model;
    ph->integrator = pb.state_integrator;
    ph->k = pb.ionic_params[0];
    ph->a = pb.ionic_params[1];
    ph->eps0 = pb.ionic_params[2];
    ph->mu1 = pb.ionic_params[3];
    ph->mu2 = pb.ionic_params[4];
    ph->inv_ts = pb.ionic_params[5] > 0 ? 1.0 / pb.ionic_params[5] : 1.0;
    ph->act = pb.act_threshold;
    // Lebesgue-type bound: |phi(x_probe)| <= (max over probe tables of sum_j |l_j(rho)|)^d max|u|
    const int n = pb.order + 1;
    double lam = 0.0;
    for (int l = 0; l <= pb.max_refine; ++l)
        for (int a = 0; a < n; ++a) {
            double sabs = 0.0;
            for (int j = 0; j < n; ++j) sabs += fabs(T.pphi[l][a][j]);
            if (sabs > lam) lam = sabs;
        }
    ph->lat_gate = 0.9 * fabs(pb.act_threshold) / pow(lam, d);
}

template <typename R>
void convert_tables(const Tables<double>& a, Tables<R>* b) {
    for (int i = 0; i < 3; ++i) {
        b->bL[i] = (R)a.bL[i]; b->bR[i] = (R)a.bR[i];
        b->dL[i] = (R)a.dL[i]; b->dR[i] = (R)a.dR[i];
        b->w[i] = (R)a.w[i];
        for (int j = 0; j < 3; ++j) {
            b->D1[i][j] = (R)a.D1[i][j];
            for (int c = 0; c < 2; ++c) {
                b->Pi[c][i][j] = (R)a.Pi[c][i][j];
                b->Pd[c][i][j] = (R)a.Pd[c][i][j];
            }
        }
    }
    for (int l = 0; l < 8; ++l)
        for (int i = 0; i < 3; ++i) {
            b->pfl[l][i] = a.pfl[l][i];
            for (int j = 0; j < 3; ++j) b->pphi[l][i][j] = (R)a.pphi[l][i][j];
        }
}

template <typename R>
void convert_phys(const Phys<double>& a, Phys<R>* b) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) b->D[i][j] = (R)a.D[i][j];
    b->gamma = (R)a.gamma;
    for (int l = 0; l < 8; ++l) {
        b->Wvol[l] = (R)a.Wvol[l];
        for (int q = 0; q < 27; ++q) b->Minv[l][q] = (R)a.Minv[l][q];
        for (int k = 0; k < 3; ++k) {
            b->h[l][k] = (R)a.h[l][k];
            b->h2[l][k] = (R)a.h2[l][k];
            b->Wface[l][k] = (R)a.Wface[l][k];
            b->kfac[l][k] = a.kfac[l][k];
        }
    }
    b->k = (R)a.k; b->a = (R)a.a; b->eps0 = (R)a.eps0; b->mu1 = (R)a.mu1; b->mu2 = (R)a.mu2;
    b->inv_ts = (R)a.inv_ts;
    b->ionic = a.ionic;
    b->integrator = a.integrator;
    b->act = (R)a.act;
    b->lat_gate = (R)a.lat_gate;
}

template void convert_tables<float>(const Tables<double>&, Tables<float>*);
template void convert_tables<double>(const Tables<double>&, Tables<double>*);
template void convert_phys<float>(const Phys<double>&, Phys<float>*);
template void convert_phys<double>(const Phys<double>&, Phys<double>*);

namespace {

// Own-DOF blocks of one level: the volume block and, for every face f and kind,
// that face's own-side block (the own block of an element is their sum, the
// element operator being linear in the face terms).
template <int DIM, int P>
void level_blocks_t(const Tables<double>& T, const Phys<double>& ph, int level, double* vol,
                    double* face /* [2DIM][4][NP][NP] */) {
    constexpr int NP = Shape<DIM, P>::NP, NSUB = Shape<DIM, P>::NSUB;
    for (int j = 0; j < NP; ++j) {
        double u[NP], r[NP];
        for (int q = 0; q < NP; ++q) u[q] = (q == j) ? 1.0 : 0.0;
        for (int q = 0; q < NP; ++q) r[q] = 0.0;
        volume_term<double, DIM, P>(T, ph, level, u, r);
        for (int q = 0; q < NP; ++q) vol[q * NP + j] = r[q];
        for (int f = 0; f < 2 * DIM; ++f) {
            const int k = f / 2, s = (f & 1) ? 1 : -1;
            for (int kd = 0; kd < 4; ++kd) {
                for (int q = 0; q < NP; ++q) r[q] = 0.0;
                if (kd == 1) face_term_own<double, DIM, P>(T, ph, k, s, level, -1, u, level, level, r);
                else if (kd == 2 && level > 0)
                    face_term_own<double, DIM, P>(T, ph, k, s, level, -1, u, level - 1, level, r);
                else if (kd == 3 && level < 7)
                    for (int sb = 0; sb < NSUB; ++sb)
                        face_term_own<double, DIM, P>(T, ph, k, s, level, sb, u, level + 1, level + 1, r);
                double* F = face + ((size_t)(f * 4 + kd) * NP) * NP;
                for (int q = 0; q < NP; ++q) F[q * NP + j] = r[q];
            }
        }
    }
}

}  // namespace

void level_blocks(const Tables<double>& T, const Phys<double>& ph, int dim, int p, int level,
                  std::vector<double>* vol, std::vector<double>* face) {
    const int NP = (dim == 2) ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1);
    vol->assign((size_t)NP * NP, 0.0);
    face->assign((size_t)2 * dim * 4 * NP * NP, 0.0);
    if (dim == 2 && p == 1) level_blocks_t<2, 1>(T, ph, level, vol->data(), face->data());
    else if (dim == 2 && p == 2) level_blocks_t<2, 2>(T, ph, level, vol->data(), face->data());
    else if (dim == 3 && p == 1) level_blocks_t<3, 1>(T, ph, level, vol->data(), face->data());
    else level_blocks_t<3, 2>(T, ph, level, vol->data(), face->data());
}

double class_cfl_from_blocks(const Tables<double>& T, const Phys<double>& ph, int dim, int p, int level,
                             unsigned cfg, const std::vector<double>& vol, const std::vector<double>& face) {
    const int n1 = p + 1;
    const int NP = (dim == 2) ? n1 * n1 : n1 * n1 * n1;
    std::vector<double> B(vol);
    for (int f = 0; f < 2 * dim; ++f) {
        const int kd = (cfg >> (2 * f)) & 3;
        const double* F = face.data() + ((size_t)(f * 4 + kd) * NP) * NP;
        for (int i = 0; i < NP * NP; ++i) B[i] += F[i];
    }
    double worst = 0.0;
    for (int i = 0; i < NP; ++i) {
        double Mi = ph.Wvol[level];
        int r = i;
        for (int k = 0; k < dim; ++k) {
            Mi *= T.w[r % n1];
            r /= n1;
        }
        double row = 0.0;
        for (int j = 0; j < NP; ++j) row += fabs(B[i * NP + j]) / Mi;
        if (row > worst) worst = row;
    }
    return 1.0 / worst;
}

double class_cfl(const Tables<double>& T, const Phys<double>& ph, int dim, int p, int level,
                 unsigned cfg) {
    std::vector<double> vol, face;
    level_blocks(T, ph, dim, p, level, &vol, &face);
    return class_cfl_from_blocks(T, ph, dim, p, level, cfg, vol, face);
}

namespace {

template <int DIM>
void q1_blocks_t(const Tables<double>& T, const Phys<double>& ph, int L, std::vector<double>* vol,
                 std::vector<double>* face, std::vector<double>* kelly) {
    using S = Shape<DIM, 1>;
    constexpr int NP = S::NP, NF = S::NF, NSUB = S::NSUB, NT = S::NT;
    constexpr int NREL = 1 + 2 * NSUB;
    vol->assign((size_t)8 * NP * NP, 0.0);
    face->assign((size_t)NF * 8 * NREL * 2 * NP * NP, 0.0);
    kelly->assign((size_t)NF * 8 * NREL * 2 * NT * NP, 0.0);
    double zero[NP] = {0};
    for (int l = 0; l < 8; ++l) {
        for (int j = 0; j < NP; ++j) {
            double u[NP] = {0}, r[NP] = {0};
            u[j] = 1.0;
            volume_term<double, DIM, 1>(T, ph, l, u, r);
            for (int q = 0; q < NP; ++q) (*vol)[((size_t)l * NP + q) * NP + j] = r[q];
        }
        for (int f = 0; f < NF; ++f) {
            const int k = f / 2, s = (f & 1) ? 1 : -1;
            for (int rel = 0; rel < NREL; ++rel) {
                int lo = l, ln, lf, cb_own, cb_nb;
                if (rel == 0) {
                    ln = l; lf = l; cb_own = -1; cb_nb = -1;
                } else if (rel <= NSUB) {
                    if (l == 0) continue;
                    ln = l - 1; lf = l; cb_own = -1; cb_nb = rel - 1;
                } else {
                    if (l >= 7) continue;
                    ln = l + 1; lf = l + 1; cb_own = rel - 1 - NSUB; cb_nb = -1;
                }
                const size_t fb = (((size_t)f * 8 + l) * NREL + rel) * 2;
                for (int side = 0; side < 2; ++side)
                    for (int j = 0; j < NP; ++j) {
                        double e[NP] = {0}, r[NP] = {0};
                        e[j] = 1.0;
                        const double* own = side == 0 ? e : zero;
                        const double* nb = side == 0 ? zero : e;
                        face_term<double, DIM, 1>(T, ph, k, s, lo, cb_own, own, ln, cb_nb, nb, lf, r);
                        for (int q = 0; q < NP; ++q) (*face)[((fb + side) * NP + q) * NP + j] = r[q];
                        // Kelly: flux jump at the face points, scaled by sqrt(h_F/(2p) W_t) W_F
                        double vo[NT], vn[NT], go[DIM][NT], gn[DIM][NT], W[NT];
                        face_eval<double, DIM, 1>(T, ph.h2[lo], k, s, cb_own, own, vo, go);
                        face_eval<double, DIM, 1>(T, ph.h2[ln], k, -s, cb_nb, nb, vn, gn);
                        face_weights<double, DIM, 1>(T, ph, lf, k, W);
                        const double WF = ph.Wface[lf][k];
                        const double area = WF * (double)(1 << (DIM - 1));
                        const double hF = (DIM == 2) ? area : sqrt(area);
                        for (int t = 0; t < NT; ++t) {
                            double fo = 0, fn = 0;
                            for (int m = 0; m < DIM; ++m) {
                                fo += ph.D[k][m] * go[m][t];
                                fn += ph.D[k][m] * gn[m][t];
                            }
                            const double c = sqrt(hF / 2.0 * W[t]) * WF;
                            (*kelly)[((fb + side) * NT + t) * NP + j] = c * (fo - fn);
                        }
                    }
            }
        }
    }
}

}  // namespace

void q1_blocks(const Tables<double>& T, const Phys<double>& ph, int dim, int L, std::vector<double>* vol,
               std::vector<double>* face, std::vector<double>* kelly) {
    if (dim == 2) q1_blocks_t<2>(T, ph, L, vol, face, kelly);
    else q1_blocks_t<3>(T, ph, L, vol, face, kelly);
}

namespace {

// x rounded to the nearest FP16 value (11-bit significand, subnormal spacing 2^-24),
// ties to even; |x| must stay below 65520.
double round_half(double x) {
    if (x == 0.0) return 0.0;
    int ex = 0;
    frexp(x, &ex);                           // |x| in [2^(ex-1), 2^ex)
    const int e = ex - 1 < -14 ? -14 : ex - 1;   // exponent of the FP16 binade (normal or subnormal)
    return ldexp(nearbyint(ldexp(x, 10 - e)), e - 10);
}

// IEEE binary16 bit pattern of an FP16-representable value.
uint16_t half_bits(double x) {
    uint16_t sign = 0;
    if (x < 0) {
        sign = 0x8000;
        x = -x;
    }
    if (x == 0.0) return sign;
    int ex = 0;
    frexp(x, &ex);
    const int e = ex - 1;
    if (e < -14) return (uint16_t)(sign | (uint16_t)ldexp(x, 24));   // subnormal: x / 2^-24
    const uint16_t frac = (uint16_t)(ldexp(x, 10 - e) - 1024.0);
    return (uint16_t)(sign | (uint16_t)((e + 15) << 10) | frac);
}

}  // namespace

int q2_tensor_blocks(const Tables<double>& T, const Phys<double>& ph, std::vector<uint16_t>* out) {
    constexpr int NP = 27, NN = 32, KK = 192;
    std::vector<double> full((size_t)NN * KK, 0.0);
    double zero[NP] = {0};
    for (int j = 0; j < NP; ++j) {
        double u[NP] = {0};
        u[j] = 1.0;
        double r[NP] = {0};
        volume_term<double, 3, 2>(T, ph, 0, u, r);
        for (int f = 0; f < 6; ++f) {
            const int k = f / 2, s = (f & 1) ? 1 : -1;
            face_term<double, 3, 2>(T, ph, k, s, 0, -1, u, 0, -1, zero, 0, r);
        }
        for (int q = 0; q < NP; ++q) full[(size_t)q * KK + j] = r[q];
        for (int f = 0; f < 6; ++f) {
            const int k = f / 2, s = (f & 1) ? 1 : -1;
            double rn[NP] = {0};
            face_term<double, 3, 2>(T, ph, k, s, 0, -1, zero, 0, -1, u, 0, rn);
            for (int q = 0; q < NP; ++q) full[(size_t)q * KK + NP * (f + 1) + j] = rn[q];
        }
    }
    double mx = 0.0;
    for (double x : full) mx = fmax(mx, fabs(x));
    int ex = 0;
    if (mx > 0) frexp(mx, &ex);
    const int t = 15 - ex;                   // max |B| 2^t in [2^14, 2^15)
    out->assign((size_t)2 * NN * KK, 0);
    for (size_t i = 0; i < full.size(); ++i) {
        const double x = ldexp(full[i], t);
        const double hi = round_half(x);
        (*out)[i] = half_bits(hi);
        (*out)[full.size() + i] = half_bits(round_half(x - hi));
    }
    return t;
}

void q2_correction_blocks(const Tables<double>& T, const Phys<double>& ph, std::vector<float>* out) {
    constexpr int NP = 27, RS = 28, NB = 14;
    out->assign((size_t)6 * NB * NP * RS, 0.0f);
    double zero[NP] = {0};
    for (int f = 0; f < 6; ++f) {
        const int k = f / 2, s = (f & 1) ? 1 : -1;
        for (int j = 0; j < NP; ++j) {
            double u[NP] = {0};
            u[j] = 1.0;
            double blk[NB][NP] = {{0}};
            double own0[NP] = {0}, own1[NP] = {0};
            // same-level own blocks at levels 0 and 1
            face_term<double, 3, 2>(T, ph, k, s, 0, -1, u, 0, -1, zero, 0, own0);
            face_term<double, 3, 2>(T, ph, k, s, 1, -1, u, 1, -1, zero, 1, own1);
            for (int q = 0; q < NP; ++q) blk[0][q] = -own0[q];
            // coarser neighbour (own level 1, neighbour level 0), tangential position p;
            // blocks of level l are 2^-(l-1) times these, so 2x gives the level-0 equivalent
            for (int p = 0; p < 4; ++p) {
                double ro[NP] = {0}, rn[NP] = {0};
                face_term<double, 3, 2>(T, ph, k, s, 1, -1, u, 0, p, zero, 1, ro);
                face_term<double, 3, 2>(T, ph, k, s, 1, -1, zero, 0, p, u, 1, rn);
                for (int q = 0; q < NP; ++q) {
                    blk[1 + p][q] = 2.0 * (ro[q] - own1[q]);
                    blk[5 + p][q] = 2.0 * rn[q];
                }
            }
            // finer neighbours (own level 0, neighbours level 1) on subfaces sb
            for (int sb = 0; sb < 4; ++sb) {
                double ro[NP] = {0}, rn[NP] = {0};
                face_term<double, 3, 2>(T, ph, k, s, 0, sb, u, 1, -1, zero, 1, ro);
                face_term<double, 3, 2>(T, ph, k, s, 0, sb, zero, 1, -1, u, 1, rn);
                for (int q = 0; q < NP; ++q) {
                    blk[9][q] += ro[q];
                    blk[10 + sb][q] = rn[q];
                }
            }
            for (int q = 0; q < NP; ++q) blk[9][q] -= own0[q];
            for (int b = 0; b < NB; ++b)
                for (int q = 0; q < NP; ++q) (*out)[(((size_t)f * NB + b) * NP + q) * RS + j] = (float)blk[b][q];
        }
    }
}

int b_from_bound(double dt, double bound) {
    for (int b = 0; b <= 60; ++b)
        if (ldexp(dt, -b) <= bound) return b;
    return -1;
}

double auto_dt_barrier(const Tables<double>& T, const Phys<double>& ph, int dim, int p, int L, int B) {
    double cmin = INFINITY;
    const int nf = 2 * dim;
    std::vector<double> vol, face;
    for (int level = 0; level <= L; ++level) {
        level_blocks(T, ph, dim, p, level, &vol, &face);
        int choices[4], nc = 0;
        choices[nc++] = 0;
        choices[nc++] = 1;
        if (level > 0) choices[nc++] = 2;
        if (level < L) choices[nc++] = 3;
        long total = 1;
        for (int f = 0; f < nf; ++f) total *= nc;
        for (long c = 0; c < total; ++c) {
            unsigned cfg = 0;
            long r = c;
            for (int f = 0; f < nf; ++f) {
                cfg |= (unsigned)choices[r % nc] << (2 * f);
                r /= nc;
            }
            const double v = class_cfl_from_blocks(T, ph, dim, p, level, cfg, vol, face);
            if (v < cmin) cmin = v;
        }
    }
    int k = -20;
    while (ldexp(1.0, -k - B) > cmin) ++k;
    return ldexp(1.0, -k);
}

}  // namespace mdl
