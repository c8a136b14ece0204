// Instantiates the apply, DSS, geometry and layout kernels for degree 8 (n = 9).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE(9)
