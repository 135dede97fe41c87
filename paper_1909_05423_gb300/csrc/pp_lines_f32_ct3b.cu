// pp_lines_f32_ct3b.cu -- FP32 (mixed-precision) line-transform kernels for FFT lengths 192, 384, 768.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_f32_ct3b) {
  switch (a.fp.M) {
    case 192: return dispatch_io<float, float, 192>(a, oy, sin, sout, threads, st);
    case 384: return dispatch_io<float, float, 384>(a, oy, sin, sout, threads, st);
    case 768: return dispatch_io<float, float, 768>(a, oy, sin, sout, threads, st);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace pp
