// Kernels of the exchange pipeline for FFT grids of length 36 per axis.
#include "xx_launch.cuh"
XX_INSTANTIATE(36)
