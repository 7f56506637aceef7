// dp45.h -- the embedded Runge-Kutta tableaux (Dormand-Prince RK5(4)7FM and
// the other solvers of the paper's table) and the step-size controller
// constants, shared by the per-context driver (mmp.cu) and the batched
// driver (batch.cu) so that both form the same FP32 stage coefficients from
// the same FP64 step size.
#pragma once
#include <math.h>

#include <algorithm>

namespace mmp {

// Dormand and Prince (1980): a_ij (row i = stage 1..6, the last row is the
// 5th-order solution b_j), and the 4th-order weights b*_j.
constexpr double kA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
constexpr double kB4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100,
                           1.0 / 40};
// step-size controller (a reading of what the paper leaves open)
constexpr double kSafety = 0.9, kGrowMin = 0.2, kGrowMax = 5.0;

// An embedded method run as: stages 2..s, then one evaluation at the new
// (renormalised) solution, which is the first stage of the next step (for
// the FSAL methods it is their last stage).  S field evaluations per step
// after k1; row S of a is the solution weights b; e = b - b* over
// k_1 .. k_S+1; exponent = 1 / (error order + 1).
struct Tableau {
  int S;
  double a[7][7];
  double e[7];
  double exponent;
};

// The embedded solvers of the paper's table (method ids of mmp.h): Heun with
// the Euler estimate, Bogacki-Shampine 3(2), Cash-Karp 5(4), Fehlberg 5(4),
// Dormand-Prince 5(4); published tableaux, higher order propagated.
inline const Tableau& tableau(int method) {
  static const Tableau dp45 = {6,
                               {{0},
                                {1.0 / 5},
                                {3.0 / 40, 9.0 / 40},
                                {44.0 / 45, -56.0 / 15, 32.0 / 9},
                                {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729},
                                {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656},
                                {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}},
                               {35.0 / 384 - 5179.0 / 57600, 0, 500.0 / 1113 - 7571.0 / 16695,
                                125.0 / 192 - 393.0 / 640, -2187.0 / 6784 + 92097.0 / 339200,
                                11.0 / 84 - 187.0 / 2100, -1.0 / 40},
                               0.2};
  static const Tableau heun = {2, {{0}, {1.0}, {0.5, 0.5}}, {0.5 - 1.0, 0.5, 0.0}, 0.5};
  static const Tableau bs23 = {3,
                               {{0}, {0.5}, {0.0, 0.75}, {2.0 / 9, 1.0 / 3, 4.0 / 9}},
                               {2.0 / 9 - 7.0 / 24, 1.0 / 3 - 1.0 / 4, 4.0 / 9 - 1.0 / 3, -1.0 / 8},
                               1.0 / 3};
  static const Tableau cashkarp = {
      6,
      {{0},
       {1.0 / 5},
       {3.0 / 40, 9.0 / 40},
       {3.0 / 10, -9.0 / 10, 6.0 / 5},
       {-11.0 / 54, 5.0 / 2, -70.0 / 27, 35.0 / 27},
       {1631.0 / 55296, 175.0 / 512, 575.0 / 13824, 44275.0 / 110592, 253.0 / 4096},
       {37.0 / 378, 0, 250.0 / 621, 125.0 / 594, 0, 512.0 / 1771}},
      {37.0 / 378 - 2825.0 / 27648, 0, 250.0 / 621 - 18575.0 / 48384, 125.0 / 594 - 13525.0 / 55296,
       -277.0 / 14336, 512.0 / 1771 - 1.0 / 4, 0},
      0.2};
  static const Tableau rkf45 = {
      6,
      {{0},
       {1.0 / 4},
       {3.0 / 32, 9.0 / 32},
       {1932.0 / 2197, -7200.0 / 2197, 7296.0 / 2197},
       {439.0 / 216, -8.0, 3680.0 / 513, -845.0 / 4104},
       {-8.0 / 27, 2.0, -3544.0 / 2565, 1859.0 / 4104, -11.0 / 40},
       {16.0 / 135, 0, 6656.0 / 12825, 28561.0 / 56430, -9.0 / 50, 2.0 / 55}},
      {16.0 / 135 - 25.0 / 216, 0, 6656.0 / 12825 - 1408.0 / 2565, 28561.0 / 56430 - 2197.0 / 4104,
       -9.0 / 50 + 1.0 / 5, 2.0 / 55, 0},
      0.2};
  switch (method) {
    case 1: return heun;
    case 2: return bs23;
    case 3: return cashkarp;
    case 4: return rkf45;
    default: return dp45;
  }
}

// FP32 stage coefficients dt a_ij of stage i (1..S), j < i.
inline void stage_coefs(const Tableau& T, double h, int i, float* coef) {
  for (int j = 0; j < 7; ++j) coef[j] = j < i ? (float)(h * T.a[i][j]) : 0.0f;
}
// FP32 error weights in the layout of the field pass: slots j < S pair with
// the earlier stages k_1 .. k_S, slot 6 with the solution evaluation.
inline void error_coefs(const Tableau& T, double h, float* ecoef) {
  for (int j = 0; j < 7; ++j) ecoef[j] = 0.0f;
  for (int j = 0; j < T.S; ++j) ecoef[j] = (float)(h * T.e[j]);
  ecoef[6] = (float)(h * T.e[T.S]);
}
// Dormand-Prince forms (the batched driver).
inline void stage_coefs(double h, int i, float* coef) { stage_coefs(tableau(0), h, i, coef); }
inline void error_coefs(double h, float* ecoef) { error_coefs(tableau(0), h, ecoef); }
// Step-size factor of the controller.
inline double grow(double err, double tol, double exponent = 0.2) {
  double fac = err == 0.0 ? kGrowMax : kSafety * pow(tol / err, exponent);
  return std::min(std::max(fac, kGrowMin), kGrowMax);
}

}  // namespace mmp
