// tables.h -- host construction of the 1-D band tables (internal).
#pragma once
#include <vector>

namespace pint {
// q2: [4][2N+1][5] bands of M1, K1, W1, X1; q1: [4][N+1][3] (same order)
void build_level_tables(int N, double x0, double x1, std::vector<double>& q2, std::vector<double>& q1);
// G1[N+1][5], H1[N+1][5], GT[2N+1][3], HT[2N+1][3]
void build_b_tables(int N, double x0, double x1, std::vector<double>& bt);
// Convection stencils of the Sec. 5.2 two-vortex wind in skew-symmetric form
// (N - N^T)/2, node order: q2 [(2N+1)^2][25] (entry dy*5+dx couples node
// (ix, iy) to (ix+dx-2, iy+dy-2)), q1 [(N+1)^2][9] likewise with offsets -1..1.
// The wind is taken at the 4 x 4 Gauss points of each element.
void build_two_vortex_stencils(int N, double x0, double x1, std::vector<double>& q2, std::vector<double>& q1);
// The same for a caller-given wind: the Q2 interpolant of nodal values
// wind[2][(2N+1)^2] on this level's grid, taken at the same Gauss points.
void build_nodal_wind_stencils(int N, double x0, double x1, const double* wind, std::vector<double>& q2,
                               std::vector<double>& q1);
}  // namespace pint
