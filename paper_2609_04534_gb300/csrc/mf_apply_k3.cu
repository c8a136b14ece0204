// Instantiates the apply, DSS, geometry and layout kernels for degree 3 (n = 4).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE(4)
