// Step/init kernel instantiations: storage float, phase-field D3Q15;
// energy solvers RK, D3Q7, D3Q15.
#define LBM_S float
#define LBM_QH 15
#define LBM_QF_PART 0
#include "inst_step.cuh"
