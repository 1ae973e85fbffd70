// Float-float site-kernel instantiations: d_R = 7 (complex).
#include "hop_ff.cuh"

HR_FF_DEFINE(7, false, hr_ff_c7)
