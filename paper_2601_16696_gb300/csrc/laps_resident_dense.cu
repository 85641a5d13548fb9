// Resident LAPS kernels for the dense-precision Gaussian (see laps_resident.cuh).
#define LAPS_INST_KIND 4
#include "laps_resident_inst.cuh"
