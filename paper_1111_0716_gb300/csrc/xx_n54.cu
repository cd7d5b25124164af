// Kernels of the exchange pipeline for FFT grids of length 54 per axis.
#include "xx_launch.cuh"
XX_INSTANTIATE(54)
