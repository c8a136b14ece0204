// Instantiates the apply, DSS, geometry and layout kernels for degree 2 (n = 3).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE(3)
