// Instantiates the batched apply kernels of the serving loop for degree 7 (n = 8).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE_BATCH(8)
