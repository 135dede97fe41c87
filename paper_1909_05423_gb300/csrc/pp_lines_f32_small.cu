// pp_lines_f32_small.cu -- FP32 (mixed-precision) line-transform kernels for FFT lengths 64, 128 and 256.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_f32_small) {
  switch (a.fp.M) {
    case 64: return dispatch_io<float, float, 64>(a, oy, sin, sout, threads, st);
    case 128: return dispatch_io<float, float, 128>(a, oy, sin, sout, threads, st);
    case 256: return dispatch_io<float, float, 256>(a, oy, sin, sout, threads, st);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace pp
