// Resident LAPS kernels for the banana target (see laps_resident.cuh).
#define LAPS_INST_KIND 1
#include "laps_resident_inst.cuh"
