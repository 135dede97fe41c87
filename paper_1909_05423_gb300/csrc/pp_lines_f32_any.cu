// pp_lines_f32_any.cu -- FP32 (mixed-precision) line-transform kernels for any FFT length (read at run time).
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_f32_any) { return dispatch_io<float, float, 0>(a, oy, sin, sout, threads, st); }
}  // namespace pp
