// Float-float site-kernel instantiations: d_R = 8 (complex).
#include "hop_ff.cuh"

HR_FF_DEFINE(8, false, hr_ff_c8)
