// The resident solve, operator apply and allocation-free solve instantiated for one
// inner precision (FP64); the code is in solver_impl.cuh.
#define MLMC_SOLVER_PREC 0
#include "solver_impl.cuh"
