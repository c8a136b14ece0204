// Instantiates the batched apply kernels of the serving loop for degree 8 (n = 9).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE_BATCH(9)
