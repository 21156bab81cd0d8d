// Step/init kernel instantiations: storage double, phase-field D3Q15.
#define LBM_S double
#define LBM_QH 15
#include "inst_step.cuh"
