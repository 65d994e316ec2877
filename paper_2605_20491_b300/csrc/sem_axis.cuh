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

// The Hermite spectral axis on R (the appendix's discretisation): ts_plan_desc.order = -1.
constexpr int ORDER_HERMITE = -1;
constexpr int HERMITE_MAX_N = 2048;  // the O(n^3) host assembly of -B^2 bounds it
struct HermiteAxis {
  int n = 0;
  std::vector<double> x;      // Gauss-Hermite nodes, ascending
  std::vector<double> log_w;  // log of W_j = 1 / (n psi_{n-1}(x_j)^2), the Gauss weights of Hermite functions
                              // (between ~0.05 and ~0.8: every node lies where psi_{n-1} oscillates)
  std::vector<double> hs0;    // -B^2 = W^{1/2} (-D^2) W^{-1/2}, symmetric n x n row-major
};
void hermite_nodes(int n, double* x);
ts_status hermite_axis_build(int n, HermiteAxis* out);

void gll_rule(int k, std::vector<double>* xi, std::vector<double>* w);
void gll_diff_matrix(const std::vector<double>& xi, std::vector<double>* D);
// Needs k >= 1 and (n + 1) % k == 0; else TS_ERR_INVALID_ARG.
ts_status sem_axis_build(int n, double L, int k, SemAxis* out);
// Node coordinates x and weights m (may be NULL) of an axis: order 0 / 1, the uniform
// interior nodes x_i = -L + (i+1) h with m = h; order >= 2, the GLL nodes of the Q^order
// elements with their lumped masses; ORDER_HERMITE, the Gauss-Hermite nodes with the Gauss
// weights of Hermite functions.
ts_status grid_nodes_host(int n, double L, int order, double* x, double* m);

}  // namespace ts
