// pp_zmul.cuh -- products with the Thomas multipliers of the z solves.
//
// The multipliers w_k = h2 / m_k of a z system lie in (-1, 0).  For the weakly diagonally dominant
// modes (the low (kx, ky) pairs of long lines, and the pinned singular mode, whose multipliers are
// about -k/(k+1)) they approach -1, and the solution depends on 1 + w_k, which is then of the order
// of the square root of the mode's smallest eigenvalue: a double-float w_k (48 bits relative to 1)
// would carry 1 + w_k with a relative error of 2^-48 / (1 + w_k), accumulated coherently over the
// rows.  Such modes (flag ZF_NEAR1) store v_k = 1 + w_k instead, exact to its own 48 bits, and every
// product with w_k is formed from v_k:  x w = x v - x,  g - w u = (g + u) - v u,  x (-w) = x - x v.
#pragma once
#include "pp_arith.cuh"

namespace pp {

// In the N1 forms the intermediate product and sum stay unnormalised (exact leading parts, the
// error terms collected in the low part); the final sum normalises.
// x w_k for the stored multiplier v (N1: v = 1 + w_k)
template <bool N1> __device__ __forceinline__ df zw_mul(df x, df v) {
  if constexpr (N1) return mul_u(x, v) - x;
  else return x * v;
}
// g - w_k u
template <bool N1> __device__ __forceinline__ df zw_sub(df g, df v, df u) {
  if constexpr (N1) return add_u(g, u) - mul_u(v, u);
  else return g - v * u;
}
// x (-w_k), the coefficient of the first-order recurrences of the factorisation
template <bool N1> __device__ __forceinline__ df zw_neg_mul(df x, df v) {
  if constexpr (N1) return x - mul_u(x, v);
  else return x * (-v);
}

}  // namespace pp
