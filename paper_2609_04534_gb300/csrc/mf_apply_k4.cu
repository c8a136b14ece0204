// Instantiates the apply, DSS, geometry and layout kernels for degree 4 (n = 5).
#include "mf_kernels.cuh"
MF_INSTANTIATE_DEGREE(5)
