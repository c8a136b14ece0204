// Instantiates the batched apply kernels of the serving loop for degree 1 (n = 2).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE_BATCH(2)
