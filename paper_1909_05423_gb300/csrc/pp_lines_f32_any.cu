// pp_lines_f32_any.cu -- FP32 (mixed-precision) line-transform kernels for run-time FFT lengths with
// radices 2, 3, 4 and 8.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_f32_any) { return dispatch_io<float, float, 0>(a, oy, sin, sout, threads, st); }
}  // namespace pp
