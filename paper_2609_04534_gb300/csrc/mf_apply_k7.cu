// Instantiates the apply, DSS, geometry and layout kernels for degree 7 (n = 8).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE(8)
