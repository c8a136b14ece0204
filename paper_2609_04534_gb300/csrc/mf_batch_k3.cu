// Instantiates the batched apply kernels of the serving loop for degree 3 (n = 4).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE_BATCH(4)
