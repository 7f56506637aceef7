// dp45.h -- the Dormand-Prince RK5(4)7FM tableau (FSAL, local extrapolation)
// and the step-size controller constants, shared by the per-context driver
// (mmp.cu) and the batched driver (batch.cu) so that both form the same
// FP32 stage coefficients from the same FP64 step size.
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
constexpr double kSafety = 0.9, kGrowMin = 0.2, kGrowMax = 5.0, kExponent = 0.2;

// FP32 stage coefficients dt a_ij of stage i (1..6), j < i.
inline void stage_coefs(double h, int i, float* coef) {
  for (int j = 0; j < 7; ++j) coef[j] = j < i ? (float)(h * kA[i][j]) : 0.0f;
}
// FP32 error weights dt (b_j - b*_j), j = 0..6.
inline void error_coefs(double h, float* ecoef) {
  for (int j = 0; j < 7; ++j) ecoef[j] = (float)(h * ((j < 6 ? kA[6][j] : 0.0) - kB4[j]));
}
// Step-size factor of the controller.
inline double grow(double err, double tol) {
  double fac = err == 0.0 ? kGrowMax : kSafety * pow(tol / err, kExponent);
  return std::min(std::max(fac, kGrowMin), kGrowMax);
}

}  // namespace mmp
