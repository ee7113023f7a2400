// yz-pass kernels, double arithmetic, operator format 2 (0 plain, 1 Tucker-like, 2 TT-like).
#include "yz_dispatch.cuh"

FMM_YZ_UNIT(double, f64, 2)
