// pp_lines_f32_large.cu -- FP32 (mixed-precision) line-transform kernels for FFT lengths 512 and 1024.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_f32_large) {
  switch (a.fp.M) {
    case 512: return dispatch_io<float, float, 512>(a, oy, sin, sout, threads, st);
    case 1024: return dispatch_io<float, float, 1024>(a, oy, sin, sout, threads, st);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace pp
