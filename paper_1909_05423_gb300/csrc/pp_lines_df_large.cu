// pp_lines_df_large.cu -- double-float (FP64-class) line-transform kernels for FFT lengths 512 and 1024.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_df_large) {
  switch (a.fp.M) {
    case 512: return dispatch_io<df, float2, 512>(a, oy, sin, sout, threads, st);
    case 1024: return dispatch_io<df, float2, 1024>(a, oy, sin, sout, threads, st);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace pp
