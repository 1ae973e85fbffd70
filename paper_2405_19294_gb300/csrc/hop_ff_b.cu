// Float-float site-kernel instantiations: d_R = 5 (complex), d_R = 6 (complex).
#include "hop_ff.cuh"

HR_FF_DEFINE(5, false, hr_ff_c5)
HR_FF_DEFINE(6, false, hr_ff_c6)
