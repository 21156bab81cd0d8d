// Step/init kernel instantiations: storage double, phase-field D3Q15;
// energy solvers RK, D3Q7, D3Q15.
#define LBM_S double
#define LBM_QH 15
#define LBM_QF_PART 0
#include "inst_step.cuh"
