// pp_range.cuh -- range report of the kernels that solve along z (tridiagonal sweeps, or the
// diagonal solve of periodic z by transform).
//
// The spill and the double-float pairs have FP32's exponent range.  Every thread keeps the
// largest |value| of the scaled right-hand sides it reads and of the solutions it writes; the
// blocks reduce them into two plan-owned words, and the last block of the launch sets the plan's
// range bit when the largest scaled input lies below dmin = 2^-100 (then the low parts, 2^-24
// below, are subnormal and the solve loses accuracy norm-wise), or the largest output is above
// umax (the inverse transforms, which sum up to 2 nx and 2 ny values, and nz for the inverse z
// transform, may overflow), or a value is not finite.  The decision is per launch and on the
// largest magnitudes only, so tiny values beside large ones (the tails of a Gaussian source)
// never raise it.
#pragma once
#include "pp_internal.h"

namespace pp {

// m = max(m, |v|) propagating NaN (max.NaN), one FMNMX per tracked value
__device__ __forceinline__ void track(float& m, float v) {
  asm("max.NaN.f32 %0, %0, %1;" : "+f"(m) : "f"(fabsf(v)));
}
__device__ __forceinline__ float max_nan(float a, float b) {
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// Block reduction of the two maxima (blocks of at most 1024 threads, every thread calls it) and
// the per-launch decision of the last block.  rstat: [0] status bits, [1] / [2] running maxima
// (FP32 bits), [3] count of finished blocks; nblocks: blocks of the launch.
__device__ __forceinline__ void range_report(unsigned* rstat, float dmin, float umax_lim, unsigned nblocks,
                                             float dmax, float umax) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dmax = max_nan(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    umax = max_nan(umax, __shfl_xor_sync(0xffffffffu, umax, o));
  }
  __shared__ float s_d[32], s_u[32];
  const int w = (int)threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { s_d[w] = dmax; s_u[w] = umax; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  float D = s_d[0], U = s_u[0];
  for (int i = 1; i < ((int)blockDim.x + 31) / 32; i++) { D = max_nan(D, s_d[i]); U = max_nan(U, s_u[i]); }
  // non-negative floats and NaN order as their bit patterns (sign cleared)
  const unsigned db = __float_as_uint(D) & 0x7fffffffu, ub = __float_as_uint(U) & 0x7fffffffu;
  unsigned* r = rstat;
  if (db > *reinterpret_cast<volatile unsigned*>(r + 1)) atomicMax(r + 1, db);
  if (ub > *reinterpret_cast<volatile unsigned*>(r + 2)) atomicMax(r + 2, ub);
  __threadfence();
  if (atomicAdd(r + 3, 1u) == nblocks - 1) {
    // last block: every other block fenced its maxima before counting itself
    __threadfence();
    const float Dt = __uint_as_float(atomicExch(r + 1, 0u)), Ut = __uint_as_float(atomicExch(r + 2, 0u));
    atomicExch(r + 3, 0u);
    const bool bad = !(Dt <= 3.4e38f) || !(Ut <= umax_lim) || (Dt > 0.0f && Dt < dmin);  // NaN fails <=
    if (bad) atomicOr(r, kStatusRange);
  }
}

}  // namespace pp
