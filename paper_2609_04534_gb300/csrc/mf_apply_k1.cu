// Instantiates the apply, DSS, geometry and layout kernels for degree 1 (n = 2).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE(2)
