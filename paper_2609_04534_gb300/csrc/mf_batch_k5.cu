// Instantiates the batched apply kernels of the serving loop for degree 5 (n = 6).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE_BATCH(6)
