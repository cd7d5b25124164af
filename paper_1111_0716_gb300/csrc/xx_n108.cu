// Kernels of the exchange pipeline for FFT grids of length 108 per axis.
#include "xx_launch.cuh"
XX_INSTANTIATE(108)
