// FP64 instantiation of the step and rebuild kernels.
#include "md_kernels.cuh"

#define REAL double
#include "md_launch.inc"
#undef REAL
