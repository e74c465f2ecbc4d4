// The resident solve, operator apply and allocation-free solve instantiated for one
// inner precision (BF16 storage); the code is in solver_impl.cuh.
#define MLMC_SOLVER_PREC 2
#include "solver_impl.cuh"
