// pp_lines_df_small.cu -- double-float (FP64-class) line-transform kernels for FFT lengths 64, 128 and 256.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_df_small) {
  switch (a.fp.M) {
    case 64: return dispatch_io<df, float2, 64>(a, oy, sin, sout, threads, st);
    case 128: return dispatch_io<df, float2, 128>(a, oy, sin, sout, threads, st);
    case 256: return dispatch_io<df, float2, 256>(a, oy, sin, sout, threads, st);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace pp
