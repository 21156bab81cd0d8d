// Step/init kernel instantiations: storage double, phase-field D3Q27.
#define LBM_S double
#define LBM_QH 27
#include "inst_step.cuh"
