// Instantiation of the 3D stage kernels in the float bulk type for N = 2..5.
#include "dgk_launch.cuh"

DGK_DEFINE_TABLE(dgk_table_3d_f32, 3, float)
