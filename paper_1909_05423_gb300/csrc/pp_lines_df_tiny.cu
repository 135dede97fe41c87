// pp_lines_df_tiny.cu -- double-float (FP64-class) line-transform kernels for FFT lengths 8, 16 and 32.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_df_tiny) {
  switch (a.fp.M) {
    case 8: return dispatch_io<df, float2, 8>(a, oy, sin, sout, threads, st);
    case 16: return dispatch_io<df, float2, 16>(a, oy, sin, sout, threads, st);
    case 32: return dispatch_io<df, float2, 32>(a, oy, sin, sout, threads, st);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace pp
