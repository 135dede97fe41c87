// pp_lines.cu -- launcher of the batched line transforms (kernels in pp_lines.cuh).  Power-of-two
// FFT lengths 8..1024 use kernels compiled for that length; other lengths use the kernels that
// read the length at run time.
#include "pp_lines.cuh"

namespace pp {

cudaError_t launch_lines_impl(const LineArgs& a, bool df_arith, int oy, int sin, int sout, int threads,
                              cudaStream_t st) {
  const int M = a.fp.M;
  const bool tiny = ct_length(M) && M <= 32, small = ct_length(M) && M >= 64 && M <= 256,
             large = ct_length(M) && M >= 512;
  bool r57 = false;  // run-time length with radix-5/7 stages: the kernels that carry those butterflies
  for (int i = 0; i < a.fp.nst; i++) r57 |= (a.fp.rad[i] == 5 || a.fp.rad[i] == 7);
  if (df_arith) {
    if (tiny) return lines_df_tiny(a, oy, sin, sout, threads, st);
    if (small) return lines_df_small(a, oy, sin, sout, threads, st);
    if (large) return lines_df_large(a, oy, sin, sout, threads, st);
    return r57 ? lines_df_any57(a, oy, sin, sout, threads, st) : lines_df_any(a, oy, sin, sout, threads, st);
  }
  if (tiny) return lines_f32_tiny(a, oy, sin, sout, threads, st);
  if (small) return lines_f32_small(a, oy, sin, sout, threads, st);
  if (large) return lines_f32_large(a, oy, sin, sout, threads, st);
  return r57 ? lines_f32_any57(a, oy, sin, sout, threads, st) : lines_f32_any(a, oy, sin, sout, threads, st);
}

}  // namespace pp
