// Instantiation of the 3D curved-element stage kernels in the double bulk type for N = 2..5.
#include "dgk_curved.cuh"

DGK_DEFINE_CURVED_TABLE(dgk_ctable_3d_f64, 3, double)
