// mdl_tables.h -- host construction of basis tables, physics constants and CFL classes.
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/mdl.h"
#include "mdl_element.cuh"

namespace mdl {

// Nodes and weights of the (p+1)-point Gauss-Legendre rule on [-1, 1] (p = 1, 2).
void gl_nodes(int p, double* x, double* w);
// Basis tables of the (p+1)-point GL Lagrange basis (p = 1, 2), closed-form nodes.
void make_tables(int p, Tables<double>* T);
// Physics: D = (sigma_t I + (sigma_l - sigma_t) f f^T) / (chi C_m), per-level geometry,
// Aliev-Panfilov constants, activation threshold and probe gate.
void make_phys(const mdl_problem& pb, const Tables<double>& T, Phys<double>* ph);

template <typename R>
void convert_tables(const Tables<double>& a, Tables<R>* b);
template <typename R>
void convert_phys(const Phys<double>& a, Phys<R>* b);

// Gershgorin bound CFL_e = 1 / max_i (|L_ii| + sum_{j != i} |L_ij|), L = M^-1 K_e,
// with K_e the element's own diagonal block of K = -A (Eq. cfl-monodomain), for an
// element of `level` whose faces have kinds cfg (2 bits per face, FaceKind).
double class_cfl(const Tables<double>& T, const Phys<double>& ph, int dim, int p, int level,
                 unsigned cfg);
// Per-level volume block and per (face, kind) own-side face blocks; the own block of a
// class is vol + sum_f face[f][kind_f].
void level_blocks(const Tables<double>& T, const Phys<double>& ph, int dim, int p, int level,
                  std::vector<double>* vol, std::vector<double>* face);
double class_cfl_from_blocks(const Tables<double>& T, const Phys<double>& ph, int dim, int p, int level,
                             unsigned cfg, const std::vector<double>& vol, const std::vector<double>& face);

// Smallest b >= 0 with dt 2^-b <= bound; -1 if none below 60.
int b_from_bound(double dt, double bound);

// Q1 class blocks.  Every Q1 face contribution to an element's residual is the linear
// map r += A_own u + A_nb u_nb; it depends only on (face f, own level l, relation rel),
// rel = 0 same level, 1 + pos coarser neighbour (pos = tangential position bits),
// 1 + 2^(d-1) + sub finer neighbour on subface sub.  Tables (row-major NP x NP blocks):
//   vol [8][NP][NP], face [NF][8][NREL][2][NP][NP] (0 own, 1 neighbour),
//   kelly [NF][8][NREL][2][NT][NP]: sqrt(c_t) times the flux jump at face point t, so
//   that a face's Kelly contribution is sum_t (K_own u + K_nb u_nb)_t^2.
void q1_blocks(const Tables<double>& T, const Phys<double>& ph, int dim, int L, std::vector<double>* vol,
               std::vector<double>* face, std::vector<double>* kelly);

// Q2 3D level-0 operator of the tensor-core sweep as two FP16 terms (binary16 bit
// patterns, out = [hi | lo], each 32 x 192 row-major), scaled by 2^t with t returned:
// row q = output DOF (27 used), columns 27 s + j: s = 0 the own block A_vol + sum_f A_own,f
// (same-level neighbours on all six faces), s = 1 + f the same-level neighbour block of
// face f.  Blocks of level l are 2^-l times these (box elements).
int q2_tensor_blocks(const Tables<double>& T, const Phys<double>& ph, std::vector<uint16_t>* out);

// Q2 3D blocks that turn the tensor product of an element with non-regular faces into its
// exact residual, FP32 [6 faces][14][27 rows][28 (27 used)], level-0 equivalents (level l:
// 2^-l times these): 0 boundary face (-A_own,same); 1+p coarser neighbour at tangential
// position p: own block minus A_own,same; 5+p its neighbour block; 9 finer neighbours: the
// own blocks of the four subfaces minus A_own,same; 10+sb neighbour block of subface sb.
void q2_correction_blocks(const Tables<double>& T, const Phys<double>& ph, std::vector<float>* out);

// Largest 2^-k with 2^-k 2^-B <= min over all admissible classes (levels 0..L).
double auto_dt_barrier(const Tables<double>& T, const Phys<double>& ph, int dim, int p, int L, int B);

}  // namespace mdl
