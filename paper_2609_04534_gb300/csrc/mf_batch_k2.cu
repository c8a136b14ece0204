// Instantiates the batched apply kernels of the serving loop for degree 2 (n = 3).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE_BATCH(3)
