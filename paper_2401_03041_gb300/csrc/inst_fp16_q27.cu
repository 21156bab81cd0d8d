// Step/init kernel instantiations: storage __half, phase-field D3Q27.
#define LBM_S __half
#define LBM_QH 27
#include "inst_step.cuh"
