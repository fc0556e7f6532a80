// mdl_tables.h -- host construction of basis tables, physics constants and CFL classes.
#pragma once

#include <vector>

#include "../../include/mdl.h"
#include "mdl_element.cuh"

namespace mdl {

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

// Largest 2^-k with 2^-k 2^-B <= min over all admissible classes (levels 0..L).
double auto_dt_barrier(const Tables<double>& T, const Phys<double>& ph, int dim, int p, int L, int B);

}  // namespace mdl
