// Instantiates the batched apply kernels of the serving loop for degree 4 (n = 5).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE_BATCH(5)
