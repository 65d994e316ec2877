// One axis of the Q^k spectral element discretisation: see sem_axis.cu.
#pragma once
#include <vector>

#include "common.cuh"

namespace ts {

struct SemAxis {
  int n = 0, k = 0;
  std::vector<double> x;      // interior node coordinates, n
  std::vector<double> m;      // lumped mass (diagonal of M), n
  std::vector<double> stiff;  // assembled stiffness restricted to the interior, n x n row-major
};

void gll_rule(int k, std::vector<double>* xi, std::vector<double>* w);
void gll_diff_matrix(const std::vector<double>& xi, std::vector<double>* D);
// Needs k >= 1 and (n + 1) % k == 0; else TS_ERR_INVALID_ARG.
ts_status sem_axis_build(int n, double L, int k, SemAxis* out);
// Interior node coordinates x and lumped masses m (may be NULL) of an axis (order <= 1:
// uniform x_i = -L + (i+1) h, m = h; else the GLL nodes of the Q^order elements).
ts_status grid_nodes_host(int n, double L, int order, double* x, double* m);

}  // namespace ts
