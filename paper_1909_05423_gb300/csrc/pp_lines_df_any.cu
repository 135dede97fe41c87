// pp_lines_df_any.cu -- double-float (FP64-class) line-transform kernels for run-time FFT lengths
// with radices 2, 3, 4 and 8.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_df_any) { return dispatch_io<df, float2, 0>(a, oy, sin, sout, threads, st); }
}  // namespace pp
