// pp_lines_f32_ct3a.cu -- FP32 (mixed-precision) line-transform kernels for FFT lengths 24, 48, 96.
#include "pp_lines.cuh"

namespace pp {
PP_LINES_GROUP_DECL(lines_f32_ct3a) {
  switch (a.fp.M) {
    case 24: return dispatch_io<float, float, 24>(a, oy, sin, sout, threads, st);
    case 48: return dispatch_io<float, float, 48>(a, oy, sin, sout, threads, st);
    case 96: return dispatch_io<float, float, 96>(a, oy, sin, sout, threads, st);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace pp
