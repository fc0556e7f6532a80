// mdl_geometry.h -- curved (mapped) meshes: the map from the reference box to the physical
// domain and the per-element geometric factors of the SIPG operator on it (host, FP64).
//
// The forest lives on the reference box [0, L_0] x [0, L_1] (x [0, L_2]); a smooth map
// x = Phi(X) gives the physical domain (the paper's curved ventricle meshes, Sec. 3.3).
// An element with reference lower corner X_c and extents h has the element map
// x(xi) = Phi(X_c + (xi + 1) h / 2), Jacobian J = DPhi(X) diag(h / 2).  On such an element
// the bilinear form of Eq. monodomain-primal-formulation with the flux of
// Eq. monodomain-numerical-flux, evaluated at the GL points, needs per point:
//   volume node q:  G_q = W_q |det DPhi| S DPhi^-1 D(x) DPhi^-T S (S = diag(2/h), W_q = w_q prod h/2),
//                   so that the volume part of a(u, v) is sum_q grad_xi v . G_q grad_xi u,
//                   and the GL mass M_q = W_q |det DPhi|;
//   face point t:   c = S DPhi^-1 D(x) n (n the element's outward unit normal, parallel to
//                   DPhi^-T e_k), so that n . D grad u = c . grad_xi u; the area weight
//                   dS = W_t |det DPhi| |DPhi^-T e_k| (Nanson's formula, W_t the face GL
//                   weight times the tangential h/2); and the penalty
//                   kappa = gamma n.D n |DPhi^-T e_k| / h_k (the element extent normal to
//                   the face is h_k / |DPhi^-T e_k|; both sides have the same level).
// Maps (mdl_problem.geometry): MDL_GEOMETRY_AFFINE, Phi(X) = A X + b; MDL_GEOMETRY_SHELL,
// an ellipsoidal shell sector (azimuth from X_0, polar angle from X_1 in 3D, transmural
// position from the last axis; semi-axes linear from the inner to the outer surface).
// With fibre_ref the fibre follows DPhi e_0 (the image of the first reference axis).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mdl.h"
#include "mdl_element.cuh"
#include "mdl_geofactors.cuh"

namespace mdl {

// The problem's geometry and diffusion as plain values for geo_eval / geo_element.
GeoArgs geo_args(const mdl_problem& p);

// x = Phi(X) and J = DPhi(X) (J[i][j] = d x_i / d X_j) of the problem's map; 3D layout,
// 2D uses the leading 2 x 2 block.
void geo_map(const mdl_problem& p, const double X[3], double x[3], double J[3][3]);

// Check the map's parameters (non-degenerate, orientation-preserving or reversing but
// regular on the whole reference box).  Returns MDL_OK or MDL_E_ARG with a reason.
int geo_check(const mdl_problem& p, const char** why);

// Factors of the root mesh (every element at level 0, root order: axis 0 fastest).
struct MappedFactors {
    int64_t ne = 0;
    int np = 0, nf = 0, npf = 0, ns = 0;       // nodes, faces, face points, metric entries
    std::vector<double> gvol;    // [ne][np][ns + 1]: G (xx, yy, xy | xx, yy, zz, xy, xz, yz), M_q
    std::vector<double> gface;   // [ne][nf][npf][dim + 2]: c (dim), dS, kappa (zeros on the boundary)
    std::vector<double> mass;    // [ne][np]: M_q
    std::vector<double> cfl;     // [ne]: Gershgorin bound of the element's own block (Eq. cfl-monodomain)
    std::vector<uint32_t> smask[MDL_MAX_STIM];   // [ne]: bit q if node q lies in stimulus box s
};

int mapped_factors(const mdl_problem& p, const Tables<double>& T, MappedFactors* out, std::string* err);

}  // namespace mdl
