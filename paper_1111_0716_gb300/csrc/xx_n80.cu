// Kernels of the exchange pipeline for FFT grids of length 80 per axis.
#include "xx_launch.cuh"
XX_INSTANTIATE(80)
