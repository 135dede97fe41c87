// pp_lines_df_any57.cu -- double-float line-transform kernels for run-time lengths with radix-5 or
// radix-7 stages.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_df_any57) { return dispatch_io<df, float2, -1>(a, oy, sin, sout, threads, st); }
}  // namespace pp
