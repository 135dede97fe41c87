// pp_zsolve.cu -- one tridiagonal solve along z for every (kx,ky) pair
// (Sec. "Solution of the Resulting Tridiagonal Matrices").
//
// After the x and y transforms, mode m satisfies, for k = 0..nz-1 (rows scaled by dz^2),
//     u_{k-1} + beta_m u_k + u_{k+1} = dz^2 d_k,   beta_m = -2 + dz^2 (lambda_x + lambda_y),
// with the end rows modified by the z faces (Neumann +1, Dirichlet -1 on the diagonal).
// It is solved by the Thomas algorithm with precomputed multipliers
//     w_k = 1 / (beta_k - w_{k-1})              (Toeplitz interior, Algorithm "Thomas_LowMem"),
//     g_k = (d_k - g_{k-1}) w_k,  u_k = g_k - w_k u_{k+1}.
// The multipliers depend only on the mode; they converge geometrically to a fixed point, so
// the host stores each mode's prefix up to convergence and the converged value (a few
// entries per mode on average instead of nz).  One thread owns one real component of one
// mode and streams through z; consecutive threads own consecutive components of a z-plane,
// so every load and store is coalesced.
//
// Periodic z uses the Sherman-Morrison modification (cited in the same section): with
// A = A' + u v^T, u = (gamma,0..0,1), v = (1,0..0,1/gamma),
//     x = y - c z,  y = A'^{-1} d,  z = A'^{-1} u = gamma q + p,
//     c = (y_0 + y_{n-1}/gamma) / (1 + z_0 + z_{n-1}/gamma).
// y_0 = sum_k q_k d_k (q = A'^{-1} e_0 = first row of the symmetric A'^{-1}) is accumulated in
// the forward sweep from a stored prefix of q, p = A'^{-1} e_{n-1} is generated in the
// backward sweep (p_{n-1} = w_{n-1}, p_k = -w_k p_{k+1}), so the cyclic solve also takes two
// sweeps.
//
// The singular mode of a problem without Dirichlet faces (Sec. "Well-posedness") removes the
// source mean, pins u_0 = 0, solves rows 1..n-1, and shifts the result to zero mean.
//
// All arithmetic is double-float (pp_arith.cuh), whatever the storage type of the spill.
#include "pp_internal.h"

namespace pp {

template <class S> struct ZIo;
template <> struct ZIo<float2> {
  __device__ static __forceinline__ df ld(const float2* p) { float2 v = *p; return df{v.x, v.y}; }
  __device__ static __forceinline__ void st(float2* p, df v) { *p = make_float2(v.hi, v.lo); }
};
template <> struct ZIo<float> {
  __device__ static __forceinline__ df ld(const float* p) { return df{*p, 0.0f}; }
  __device__ static __forceinline__ void st(float* p, df v) { *p = df_to_f32(v); }
};

__device__ __forceinline__ df f2df(const float* v) { return df{v[0], v[1]}; }
__device__ __forceinline__ df f2df(float2 v) { return df{v.x, v.y}; }

constexpr int ZU = 8;  // loads issued ahead in each sweep

template <class S>
__global__ void __launch_bounds__(256) k_zsolve(const ZArgs a) {
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nreal) return;
  // slot s of the (padded) spectral plane -> row, column; padding columns carry no mode
  const unsigned row = a.fd_row.div((unsigned)s);
  const int col = (int)(s - (long long)row * a.row_reals);
  if (col >= a.row_valid) return;
  const long long mi = (long long)row * a.row_modes + (a.cplx ? (col >> 1) : col);
  const ZMode m = a.modes[mi];
  S* base = reinterpret_cast<S*>(a.data) + s;
  const long long P = a.plane;
  const int n = a.nz;
  const df scale = df{a.scale[0], a.scale[1]};
  const df winf = f2df(m.winf), wlast = f2df(m.wlast);
  const float2* wt = a.wtab + m.woff;
  auto W = [&](int k) -> df {
    if (k == n - 1) return wlast;
    if (k < m.wlen) return f2df(__ldg(wt + k));
    return winf;
  };

  if (m.flags & ZF_SINGULAR) {
    // mean of the source
    df sum = df{0.f, 0.f};
    for (int k = 0; k < n; k++) sum = sum + ZIo<S>::ld(base + k * P);
    df mean = sum * df_rcp(df{(float)n, 0.f});
    // rows 1..n-1 of the pinned system (u_0 = 0); multipliers of the sub-system in the table
    df g = df{0.f, 0.f};
    for (int k = 1; k < n; k++) {
      df d = (ZIo<S>::ld(base + k * P) - mean) * scale;
      df w = f2df(__ldg(wt + (k - 1)));
      g = (d - g) * w;
      ZIo<S>::st(base + k * P, g);
    }
    df u = df{0.f, 0.f};
    df usum = df{0.f, 0.f};
    for (int k = n - 1; k >= 1; k--) {
      df gk = ZIo<S>::ld(base + k * P);
      df w = f2df(__ldg(wt + (k - 1)));
      u = (k == n - 1) ? gk : gk - w * u;
      usum = usum + u;
      ZIo<S>::st(base + k * P, u);
    }
    df umean = usum * df_rcp(df{(float)n, 0.f});
    ZIo<S>::st(base, -umean);
    for (int k = 1; k < n; k++) ZIo<S>::st(base + k * P, ZIo<S>::ld(base + k * P) - umean);
    return;
  }

  const bool periodic = (m.flags & ZF_PERIODIC) != 0;
  const float2* qt = a.qtab + m.qoff;
  const int qlen = m.qlen;

  if (!a.transpose || periodic) {
    // forward elimination g_k = (s d_k - g_{k-1}) w_k; periodic: y0 = sum q_k s d_k
    df g = df{0.f, 0.f};
    df y0 = df{0.f, 0.f};
    for (int k0 = 0; k0 < n; k0 += ZU) {
      df dv[ZU];
#pragma unroll
      for (int u = 0; u < ZU; u++)
        if (k0 + u < n) dv[u] = ZIo<S>::ld(base + (k0 + u) * P);
#pragma unroll
      for (int u = 0; u < ZU; u++) {
        int k = k0 + u;
        if (k < n) {
          df d = dv[u] * scale;
          g = (d - g) * W(k);
          if (periodic && k < qlen) y0 = y0 + f2df(__ldg(qt + k)) * d;
          ZIo<S>::st(base + k * P, g);
        }
      }
    }
    // back substitution u_k = g_k - w_k u_{k+1}
    df c = df{0.f, 0.f}, gam = df{0.f, 0.f};
    if (periodic) {
      gam = f2df(m.gam);
      c = (y0 + g * f2df(m.igam)) * f2df(m.dsm);  // g == y_{n-1}
    }
    df u = df{0.f, 0.f};
    df p = wlast;
    for (int k0 = n - 1; k0 >= 0; k0 -= ZU) {
      df gv[ZU];
#pragma unroll
      for (int t = 0; t < ZU; t++)
        if (k0 - t >= 0) gv[t] = ZIo<S>::ld(base + (k0 - t) * P);
#pragma unroll
      for (int t = 0; t < ZU; t++) {
        int k = k0 - t;
        if (k >= 0) {
          df wk = W(k);
          u = (k == n - 1) ? gv[t] : gv[t] - wk * u;
          df outv = u;
          if (periodic) {
            if (k < n - 1) p = -(wk * p);
            df zk = p;
            if (k < qlen) zk = zk + gam * f2df(__ldg(qt + k));
            outv = u - c * zk;
          }
          ZIo<S>::st(base + k * P, outv);
        }
      }
    }
  } else {
    // transposed factorisation T^T = U^T L^T:  h_k = s d_k - w_{k-1} h_{k-1},  x_k = (h_k - x_{k+1}) w_k
    df h = df{0.f, 0.f};
    df wprev = df{0.f, 0.f};
    for (int k0 = 0; k0 < n; k0 += ZU) {
      df dv[ZU];
#pragma unroll
      for (int u = 0; u < ZU; u++)
        if (k0 + u < n) dv[u] = ZIo<S>::ld(base + (k0 + u) * P);
#pragma unroll
      for (int u = 0; u < ZU; u++) {
        int k = k0 + u;
        if (k < n) {
          df d = dv[u] * scale;
          h = (k == 0) ? d : d - wprev * h;
          wprev = W(k);
          ZIo<S>::st(base + k * P, h);
        }
      }
    }
    df x = df{0.f, 0.f};
    for (int k0 = n - 1; k0 >= 0; k0 -= ZU) {
      df hv[ZU];
#pragma unroll
      for (int t = 0; t < ZU; t++)
        if (k0 - t >= 0) hv[t] = ZIo<S>::ld(base + (k0 - t) * P);
#pragma unroll
      for (int t = 0; t < ZU; t++) {
        int k = k0 - t;
        if (k >= 0) {
          x = (k == n - 1) ? hv[t] * W(k) : (hv[t] - x) * W(k);
          ZIo<S>::st(base + k * P, x);
        }
      }
    }
  }
}

cudaError_t launch_zsolve_impl(const ZArgs& a, bool df_spill, cudaStream_t st) {
  int threads = 256;
  long long grid = (a.nreal + threads - 1) / threads;
  if (df_spill) k_zsolve<float2><<<(unsigned)grid, threads, 0, st>>>(a);
  else k_zsolve<float><<<(unsigned)grid, threads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace pp
