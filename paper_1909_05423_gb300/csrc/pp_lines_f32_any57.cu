// pp_lines_f32_any57.cu -- FP32 line-transform kernels for run-time lengths with radix-5 or radix-7
// stages.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_f32_any57) { return dispatch_io<float, float, -1>(a, oy, sin, sout, threads, st); }
}  // namespace pp
