// Resident LAPS kernels for the funnel target (see laps_resident.cuh).
#define LAPS_INST_KIND 2
#include "laps_resident_inst.cuh"
