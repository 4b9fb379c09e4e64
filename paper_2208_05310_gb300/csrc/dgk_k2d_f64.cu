// Instantiation of the 2D stage kernels in the double bulk type for N = 2..5.
#include "dgk_launch.cuh"

DGK_DEFINE_TABLE(dgk_table_2d_f64, 2, double)
