// Step/init kernel instantiations: storage float, phase-field D3Q15.
#define LBM_S float
#define LBM_QH 15
#include "inst_step.cuh"
