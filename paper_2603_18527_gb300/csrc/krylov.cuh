// Interfaces shared by the Krylov solver and the solvers.
#pragma once

#include "ctx.cuh"

namespace npbs {

__global__ void k_negate(double2* y, int n);

}  // namespace npbs
