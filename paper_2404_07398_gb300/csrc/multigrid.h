// Multigrid hierarchy for the batched solver's preconditioner (host side).
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

namespace ifilt {

struct MgParams {
  int32_t coarsest_rows = 64;  // stop coarsening at or below this many rows
  int32_t max_levels = 16;
  double min_ratio = 0.8;      // stop when aggregation keeps more than this share of rows
  // Aggregation follows only strong connections |k_ij| >= strength sqrt(|k_ii k_jj|) (0: every
  // neighbour).  With strength > 0 the coarse levels also get damped-Jacobi weights scaled to
  // their operators (Galerkin masses are far from diagonal): min(2/3, (4/3) / max(lambda_max(
  // D_M^-1 M_l), lambda_max(D_K^-1 K_l))); the finest level keeps 2/3.
  double strength = 0.0;
};

// One level.  S holds the pair (K_l, M_l) on one pattern: nval = 2 per entry
// for scalar rows (k, m), 4 for 2x2-block rows (k_a, k_b, m_a, m_b); level 0
// leaves S empty (the mesh's K and lumped mass serve).  P maps level l+1 to
// level l (rows of level l), R = P^T; both have nval = 1 (scalar) or 2 (block).
struct MgHostLevel {
  int32_t n = 0;
  HostCSR S, P, R;
  std::vector<double> dk, dm;  // diagonals of K_l and M_l (real parts)
  double omega_p = 0.0;        // weight of the prolongator smoothing
  double omega_s = 2.0 / 3.0;  // damped-Jacobi weight of the smoother on this level
};

struct MgHost {
  std::vector<MgHostLevel> levels;
};

MgHost build_multigrid(const HostPrepared& h, const MgParams& prm);

}  // namespace ifilt
