// pp_lines_f32_tiny.cu -- FP32 (mixed-precision) line-transform kernels for FFT lengths 8, 16 and 32.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_f32_tiny) {
  switch (a.fp.M) {
    case 8: return dispatch_io<float, float, 8>(a, oy, sin, sout, threads, st);
    case 16: return dispatch_io<float, float, 16>(a, oy, sin, sout, threads, st);
    case 32: return dispatch_io<float, float, 32>(a, oy, sin, sout, threads, st);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace pp
