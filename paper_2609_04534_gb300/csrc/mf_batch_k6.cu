// Instantiates the batched apply kernels of the serving loop for degree 6 (n = 7).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE_BATCH(7)
