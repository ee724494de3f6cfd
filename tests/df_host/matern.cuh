// Host stand-in for the parts of csrc/matern.cuh that matern_df.cuh names:
// the lower end of the general-nu polynomials' range and the direct FP64
// evaluation (not exercised by the closed-form checks).
#pragma once
#include "matern_params.h"
namespace egs {
constexpr double kMtXlo = 1.25 * 0x1p-12;
inline double matern_eval(const egs_matern_params *, double, const double *) { return -1.0; }
}  // namespace egs
