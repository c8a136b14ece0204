// Instantiates the apply, DSS, geometry and layout kernels for degree 5 (n = 6).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE(6)
