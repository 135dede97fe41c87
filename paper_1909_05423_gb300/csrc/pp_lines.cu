// pp_lines.cu -- launcher of the batched line transforms (kernels in pp_lines.cuh).  FFT lengths
// 8..1024 that are powers of two or 3 x 2^k use kernels compiled for that length; other lengths use the kernels that
// read the length at run time.
#include "pp_lines.cuh"

namespace pp {

cudaError_t launch_lines_impl(const LineArgs& a, bool df_arith, int oy, int sin, int sout, int threads,
                              cudaStream_t st) {
  const int M = a.fp.M;
  const bool p2 = ct_length(M) && (M & (M - 1)) == 0;
  const bool tiny = p2 && M <= 32, small = p2 && M >= 64 && M <= 256, large = p2 && M >= 512;
  const bool ct3a = ct_length(M) && !p2 && M <= 96, ct3b = ct_length(M) && !p2 && M >= 192;
  bool r57 = false;  // run-time length with radix-5/7 stages: the kernels that carry those butterflies
  for (int i = 0; i < a.fp.nst; i++) r57 |= (a.fp.rad[i] == 5 || a.fp.rad[i] == 7);
  if (df_arith) {
    if (tiny) return lines_df_tiny(a, oy, sin, sout, threads, st);
    if (small) return lines_df_small(a, oy, sin, sout, threads, st);
    if (large) return lines_df_large(a, oy, sin, sout, threads, st);
    if (ct3a) return lines_df_ct3a(a, oy, sin, sout, threads, st);
    if (ct3b) return lines_df_ct3b(a, oy, sin, sout, threads, st);
    return r57 ? lines_df_any57(a, oy, sin, sout, threads, st) : lines_df_any(a, oy, sin, sout, threads, st);
  }
  if (tiny) return lines_f32_tiny(a, oy, sin, sout, threads, st);
  if (small) return lines_f32_small(a, oy, sin, sout, threads, st);
  if (large) return lines_f32_large(a, oy, sin, sout, threads, st);
  if (ct3a) return lines_f32_ct3a(a, oy, sin, sout, threads, st);
  if (ct3b) return lines_f32_ct3b(a, oy, sin, sout, threads, st);
  return r57 ? lines_f32_any57(a, oy, sin, sout, threads, st) : lines_f32_any(a, oy, sin, sout, threads, st);
}

}  // namespace pp
