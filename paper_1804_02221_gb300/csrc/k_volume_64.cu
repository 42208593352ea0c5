// Volume kernel, launch shape of 64 threads per block (k_volume.cuh).
#include "k_volume.cuh"

SWE_VOLUME_SHAPE(64)
