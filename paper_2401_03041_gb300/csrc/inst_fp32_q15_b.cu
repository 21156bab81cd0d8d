// Step/init kernel instantiations: storage float, phase-field D3Q15;
// energy solvers D3Q19, D3Q27.
#define LBM_S float
#define LBM_QH 15
#define LBM_QF_PART 1
#include "inst_step.cuh"
