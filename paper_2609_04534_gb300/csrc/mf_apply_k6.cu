// Instantiates the apply, DSS, geometry and layout kernels for degree 6 (n = 7).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE(7)
