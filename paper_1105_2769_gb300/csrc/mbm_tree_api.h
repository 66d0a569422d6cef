// Internal interface between the ABI dispatcher and the tree path.
#pragma once

#include "mbm_internal.h"

// Multi-tree approximation of Phi (Algorithm 2 with the rules of Sec. 4).
mbm_status mbm_tree_potential(mbm_ctx* ctx, const double* X, int64_t N, double eps, double alpha,
                              bool absolute, const mbm_config& cfg, mbm_tree* tree, double* phi,
                              mbm_stats* stats, cudaStream_t s);

// Tree-approximated forces F = -grad E (3 per particle, caller's order) under
// the force criterion: each component within eps S(x) + tau, S(x) the sum over
// the tuples containing x of |grad_x phi|_2 (probabilistic with alpha > 0).
mbm_status mbm_tree_forces(mbm_ctx* ctx, const double* X, int64_t N, double eps, double alpha,
                           bool absolute, const mbm_config& cfg, mbm_tree* tree, double* F3,
                           mbm_stats* stats, cudaStream_t s);

// Device bytes of one tree solve of N points (tree plus traversal scratch).
size_t mbm_tree_solve_bytes(int64_t N, const mbm_config& cfg, bool forces = false);
