// Resident LAPS kernels for the gauss target (see laps_resident.cuh).
#define LAPS_INST_KIND 0
#include "laps_resident_inst.cuh"
