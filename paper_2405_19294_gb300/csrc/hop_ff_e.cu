// Float-float site-kernel instantiations: d_R = 8 (real).
#include "hop_ff.cuh"

HR_FF_DEFINE(8, true, hr_ff_r8)
