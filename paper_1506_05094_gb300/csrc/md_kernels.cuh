// md_kernels.cuh -- all sm_103a kernels of one MD timestep (included by one translation unit per
// precision, which instantiates the templates for its Real type).
#pragma once
#include "md_rep.cuh"
