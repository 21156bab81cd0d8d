// Step/init kernel instantiations: storage double, phase-field D3Q27;
// energy solvers D3Q19, D3Q27.
#define LBM_S double
#define LBM_QH 27
#define LBM_QF_PART 1
#include "inst_step.cuh"
