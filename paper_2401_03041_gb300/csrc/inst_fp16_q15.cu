// Step/init kernel instantiations: storage __half, phase-field D3Q15.
#define LBM_S __half
#define LBM_QH 15
#include "inst_step.cuh"
