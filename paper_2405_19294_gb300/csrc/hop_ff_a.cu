// Float-float site-kernel instantiations: d_R = 2 (complex), d_R = 3 (complex), d_R = 3 (real), d_R = 4 (complex).
#include "hop_ff.cuh"

HR_FF_DEFINE(2, false, hr_ff_c2)
HR_FF_DEFINE(3, false, hr_ff_c3)
HR_FF_DEFINE(3, true, hr_ff_r3)
HR_FF_DEFINE(4, false, hr_ff_c4)
