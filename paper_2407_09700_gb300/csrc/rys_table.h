// Rys root / weight interpolation table (generated data in rys_table.cpp).
// For N = 1..RYS_NMAX roots and 0 <= T < RYS_TCUT[N], interval i = floor(RYS_SUB T) holds,
// for each root r, RYS_DEG+1 coefficients of u_r followed by RYS_DEG+1 of w_r, highest
// power first, in x = 2 (RYS_SUB T - i) - 1.  Block start:
//   RYS_COEF_OFFSET[N] + i * N * 2 * (RYS_DEG + 1).
// For T >= RYS_TCUT[N]: u_r = RYS_ASYM_U[a + r] / T and w_r = RYS_ASYM_W[a + r] / sqrt(T),
// a = RYS_ASYM_OFFSET[N].  Weights are normalised so that sum_r w_r = F_0(T).
#pragma once
#define RYS_NMAX 9
#define RYS_DEG 7
#define RYS_SUB 4
#ifdef __cplusplus
extern "C" {
#endif
extern const int RYS_TCUT[RYS_NMAX + 1];
extern const int RYS_COEF_OFFSET[RYS_NMAX + 1];
extern const int RYS_ASYM_OFFSET[RYS_NMAX + 1];
extern const int RYS_NCOEF;
extern const double RYS_COEF[];
extern const double RYS_ASYM_U[];
extern const double RYS_ASYM_W[];
#ifdef __cplusplus
}
#endif
