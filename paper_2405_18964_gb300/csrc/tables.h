// tables.h -- host construction of the 1-D band tables (internal).
#pragma once
#include <vector>

namespace pint {
// q2: [4][2N+1][5] bands of M1, K1, W1, X1; q1: [4][N+1][3] (same order)
void build_level_tables(int N, double x0, double x1, std::vector<double>& q2, std::vector<double>& q1);
// G1[N+1][5], H1[N+1][5], GT[2N+1][3], HT[2N+1][3]
void build_b_tables(int N, double x0, double x1, std::vector<double>& bt);
}  // namespace pint
