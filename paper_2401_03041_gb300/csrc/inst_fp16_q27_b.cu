// Step/init kernel instantiations: storage __half, phase-field D3Q27;
// energy solvers D3Q19, D3Q27.
#define LBM_S __half
#define LBM_QH 27
#define LBM_QF_PART 1
#include "inst_step.cuh"
