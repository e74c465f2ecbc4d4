// The resident solve, operator apply and allocation-free solve instantiated for one
// inner precision (FP32); the code is in solver_impl.cuh.
#define MLMC_SOLVER_PREC 1
#include "solver_impl.cuh"
