// Step/init kernel instantiations: storage float, phase-field D3Q27.
#define LBM_S float
#define LBM_QH 27
#include "inst_step.cuh"
