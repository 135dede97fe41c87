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
// the forward sweep from a stored prefix of q.  p = A'^{-1} e_{n-1} satisfies p_{n-1} = w_{n-1},
// p_k = -w_k p_{k+1}, so v = y - c p obeys the back substitution itself,
//     v_k = g_k - w_k v_{k+1},  v_{n-1} = g_{n-1} - c w_{n-1},
// and x_k = v_k - c gamma q_k: the cyclic solve takes the two Thomas sweeps plus the q prefix.
//
// The singular mode of a problem without Dirichlet faces (Sec. "Well-posedness") removes the
// source mean, pins u_0 = 0, solves rows 1..n-1, and shifts the result to zero mean.
//
// All arithmetic is double-float (pp_arith.cuh), whatever the storage type of the spill.
//
// Range report: see pp_range.cuh (largest scaled input and output per launch).
#include "pp_range.cuh"
#include "pp_zmul.cuh"

namespace pp {

// raw spill value -> double-float, and back
__device__ __forceinline__ df zcvt(float2 v) { return df{v.x, v.y}; }
__device__ __forceinline__ df zcvt(float v) { return df{v, 0.0f}; }
// s v for a spill value v: unnormalised (TwoProd of the leading parts plus the cross term); the
// subtraction that consumes it reads unnormalised pairs correctly
__device__ __forceinline__ df zscaled(float2 v, df s) { return mul_u(df{v.x, v.y}, s); }
__device__ __forceinline__ df zscaled(float v, df s) {
  const float p = __fmul_rn(v, s.hi);
  return df{p, __fmaf_rn(v, s.lo, __fmaf_rn(v, s.hi, -p))};
}
__device__ __forceinline__ void zput(float2* p, df v) { *p = make_float2(v.hi, v.lo); }
__device__ __forceinline__ void zput(float* p, df v) { *p = df_to_f32(v); }

__device__ __forceinline__ df f2df(const float* v) { return df{v[0], v[1]}; }
__device__ __forceinline__ df f2df(float2 v) { return df{v.x, v.y}; }

// Planes per batch.  Each sweep loads the next batch before it computes the current one, so a
// thread always has one batch of loads in flight (the sweeps are bound by loads in flight): 8
// double-float planes (64 bytes), 16 FP32 planes (64 bytes).
template <class S> struct ZBatch { static constexpr int v = (sizeof(S) == 4) ? 16 : 8; };

// raw values of planes k0 + step*u, u < ZU, that lie in [0, n)
template <int ZU, class S>
__device__ __forceinline__ void zload(S* v, const S* base, long long P, int k0, int step, int n) {
#pragma unroll
  for (int u = 0; u < ZU; u++) {
    const int k = k0 + step * u;
    if (k >= 0 && k < n) v[u] = base[(long long)k * P];
  }
}
// The same for a batch that lies wholly in [0, n), from q = base + k0 P: no tests, and each address
// one 32 x 32 -> 64-bit multiply-add of the plane stride (P32 = P < 2^31 for every plan) instead of
// a 64-bit product (the FP32-spill sweeps are bound by instruction issue).
template <int ZU, class S>
__device__ __forceinline__ void zload_full(S* v, const S* q, int P32, int step) {
#pragma unroll
  for (int u = 0; u < ZU; u++) v[u] = q[(long long)(step * u) * P32];
}
// batch loads of the sweeps: unchecked where the whole batch lies in [0, n)
template <int ZU, class S>
__device__ __forceinline__ void zload_batch(S* v, const S* base, long long P, int P32, int k0, int step, int n) {
  const int klast = k0 + step * (ZU - 1);
  if (k0 >= 0 && k0 < n && klast >= 0 && klast < n) zload_full<ZU>(v, base + (long long)k0 * P, P32, step);
  else zload<ZU>(v, base, P, k0, step, n);
}

// The singular mode: remove the source mean, pin u_0 = 0, solve rows 1..n-1, shift to zero mean.
template <class S>
__device__ __noinline__ void z_singular(S* base, long long P, int n, df scale, const float2* wt, float& dmax,
                                        float& umax) {
  // The pinned system is consistent only for a zero-mean right-hand side; a remainder c of the mean
  // would add a profile growing like c k^2 / 2.  One double-float pass leaves the rounding of a sum
  // of n values of the source's own mean magnitude (relative 2^-48 per term), so a second pass takes
  // the mean of the residuals, which are of the size of the fluctuations.
  const df rn = df_rcp(df{(float)n, 0.f});
  df sum = df{0.f, 0.f};
  for (int k = 0; k < n; k++) sum = sum + zcvt(base[k * P]);
  df mean = sum * rn;
  df rsum = df{0.f, 0.f};
  for (int k = 0; k < n; k++) rsum = rsum + (zcvt(base[k * P]) - mean);
  mean = mean + rsum * rn;
  // rows 1..n-1 of the pinned system; multipliers of the sub-system in the table
  df g = df{0.f, 0.f};
  for (int k = 1; k < n; k++) {
    df d = (zcvt(base[k * P]) - mean) * scale;
    track(dmax, d.hi);
    g = zw_mul<true>(d - g, f2df(__ldg(wt + (k - 1))));  // the pinned table is stored as 1 + w
    zput(base + k * P, g);
  }
  df u = df{0.f, 0.f};
  df usum = df{0.f, 0.f};
  for (int k = n - 1; k >= 1; k--) {
    df gk = zcvt(base[k * P]);
    u = (k == n - 1) ? gk : zw_sub<true>(gk, f2df(__ldg(wt + (k - 1))), u);
    usum = usum + u;
    zput(base + k * P, u);
  }
  df umean = usum * rn;
  // the same second pass for the solution's mean (u_0 = 0 is pinned)
  df ursum = -umean;
  for (int k = 1; k < n; k++) ursum = ursum + (zcvt(base[k * P]) - umean);
  umean = umean + ursum * rn;
  zput(base, -umean);
  track(umax, umean.hi);
  for (int k = 1; k < n; k++) {
    const df v = zcvt(base[k * P]) - umean;
    track(umax, v.hi);
    zput(base + k * P, v);
  }
}

// Steps of the Thomas recurrences, g_k = (d_k - g_{k-1}) w_k and u_k = g_k - w_k u_{k+1}.  The
// FP32-spill sweeps (mixed plans) keep their double-float pairs unnormalised: the leading parts are
// still summed and multiplied exactly and the low part collects the error terms, so a pair stays
// good to ~2^-44 of its value over the decay length of the slowest modes, while the values they
// store are rounded to FP32 anyway; the multipliers, which fix the solved matrix, keep all their
// bits.  The double-float spill (FP64-class plans) normalises every step.
template <class S, bool N1> __device__ __forceinline__ df zr_fwd(df d, df g, df w) {
  if constexpr (sizeof(S) == 4 && !N1) return mul_u(add_u(d, -g), w);
  else return zw_mul<N1>(d - g, w);
}
template <class S, bool N1> __device__ __forceinline__ df zr_bwd(df g, df w, df u) {
  if constexpr (sizeof(S) == 4 && !N1) return add_u(g, -mul_u(w, u));
  else return zw_sub<N1>(g, w, u);
}

// Two-sweep kernel: the forward sweep writes the eliminated values over the right-hand sides, the
// back substitution reads them back.  It runs for the FP32 spill (mixed plans); the double-float
// spill runs the checkpointed sweeps below, which share its arithmetic.
// MODE 0: Thomas; 1: periodic z (Sherman-Morrison); 2: transposed factorisation (adjoint).
// Batches wholly inside the converged part of the multipliers (and past the q prefix, before the
// last row) skip the per-row tests.  That is worth its extra registers where the sweeps are bound
// by instruction issue, the FP32 spill and the cyclic double-float sweeps (measured), and not in
// the Thomas double-float sweeps, which run at the copy bandwidth without it.
template <class S, int MODE> struct ZFast { static constexpr bool v = sizeof(S) == 4 || MODE == 1; };
// CTAs of 256 threads per SM the register allocation must allow (measured): 4 (64 registers)
// for the Thomas double-float sweeps, 3 (85) where the batches have a fast path, 2 for the cyclic
// FP32-spill sweeps (at 85 they spill).
template <class S, int MODE> struct ZMinBlocks {
  static constexpr int v = (MODE == 1 && sizeof(S) == 4) ? 2 : (ZFast<S, MODE>::v ? 3 : 4);
};

template <class S, int MODE, bool N1>
__device__ __forceinline__ void z_sweeps(const ZArgs& a, const ZMode& m, S* base, long long P, int n, df scale,
                                         const float2* wt, bool plus1, float& dmax, float& umax) {
  // plus1: this mode stores w itself but runs the near -1 form beside a mode of its warp that needs
  // it; its multipliers are converted to 1 + w on the fly (exact enough away from -1)
  const df one = df{1.f, 0.f};
  df winf = f2df(m.winf), wlast = f2df(m.wlast);
  if (N1 && plus1) { winf = winf + one; wlast = wlast + one; }
  const int wlen = m.wlen;
  auto W = [&](int k) -> df {
    if (k == n - 1) return wlast;
    if (k < wlen) {
      df x = f2df(__ldg(wt + k));
      if (N1 && plus1) x = x + one;
      return x;
    }
    return winf;
  };
  constexpr int ZU = ZBatch<S>::v;
  S cur[ZU], nxt[ZU];

  if constexpr (MODE != 2) {
    constexpr bool periodic = (MODE == 1);
    const float2* qt = a.qtab + m.qoff;
    const int qlen = periodic ? m.qlen : 0;
    // forward elimination g_k = (s d_k - g_{k-1}) w_k; periodic: y0 = sum q_k s d_k
    df g = df{0.f, 0.f};
    df y0 = df{0.f, 0.f};
    const int P32 = (int)P;
    zload_batch<ZU>(cur, base, P, P32, 0, 1, n);
    for (int k0 = 0; k0 < n; k0 += ZU) {
      if (k0 + ZU < n) zload_batch<ZU>(nxt, base, P, P32, k0 + ZU, 1, n);
      if (ZFast<S, MODE>::v && k0 >= wlen && k0 >= qlen && k0 + ZU < n) {
        S* const q = base + (long long)k0 * P;
#pragma unroll
        for (int u = 0; u < ZU; u++) {
          const df d = zscaled(cur[u], scale);
          track(dmax, d.hi);
          g = zr_fwd<S, N1>(d, g, winf);
          zput(q + (long long)u * P32, g);
        }
      } else {
#pragma unroll
        for (int u = 0; u < ZU; u++) {
          const int k = k0 + u;
          if (k < n) {
            df d = zscaled(cur[u], scale);
            track(dmax, d.hi);
            g = zr_fwd<S, N1>(d, g, W(k));
            if (periodic && k < qlen) y0 = y0 + f2df(__ldg(qt + k)) * d;
            zput(base + k * P, g);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < ZU; u++) cur[u] = nxt[u];
    }
    // back substitution u_k = g_k - w_k u_{k+1} (periodic: v_k, see the header)
    df c = df{0.f, 0.f}, cg = df{0.f, 0.f};
    if (periodic) {
      c = (y0 + g * f2df(m.igam)) * f2df(m.dsm);  // g == y_{n-1}
      cg = c * f2df(m.gam);
    }
    df u = df{0.f, 0.f};
    zload_batch<ZU>(cur, base, P, P32, n - 1, -1, n);
    for (int k0 = n - 1; k0 >= 0; k0 -= ZU) {
      if (k0 - ZU >= 0) zload_batch<ZU>(nxt, base, P, P32, k0 - ZU, -1, n);
      if (ZFast<S, MODE>::v && k0 - ZU + 1 >= wlen && k0 - ZU + 1 >= qlen && k0 < n - 1) {
        S* const q = base + (long long)k0 * P;
#pragma unroll
        for (int t = 0; t < ZU; t++) {
          u = zr_bwd<S, N1>(zcvt(cur[t]), winf, u);
          track(umax, u.hi);
          zput(q - (long long)t * P32, u);
        }
#pragma unroll
        for (int t = 0; t < ZU; t++) cur[t] = nxt[t];
        continue;
      }
#pragma unroll
      for (int t = 0; t < ZU; t++) {
        const int k = k0 - t;
        if (k >= 0) {
          const df gk = zcvt(cur[t]);
          if (k == n - 1) u = periodic ? zw_sub<N1>(gk, wlast, c) : gk;
          else u = zr_bwd<S, N1>(gk, W(k), u);
          df outv = u;
          if (periodic && k < qlen) outv = u - cg * f2df(__ldg(qt + k));
          track(umax, outv.hi);
          zput(base + k * P, outv);
        }
      }
#pragma unroll
      for (int t = 0; t < ZU; t++) cur[t] = nxt[t];
    }
  } else {
    // transposed factorisation T^T = U^T L^T:  h_k = s d_k - w_{k-1} h_{k-1},  x_k = (h_k - x_{k+1}) w_k
    df h = df{0.f, 0.f};
    df wprev = df{0.f, 0.f};
    const int P32 = (int)P;
    zload_batch<ZU>(cur, base, P, P32, 0, 1, n);
    for (int k0 = 0; k0 < n; k0 += ZU) {
      if (k0 + ZU < n) zload_batch<ZU>(nxt, base, P, P32, k0 + ZU, 1, n);
#pragma unroll
      for (int u = 0; u < ZU; u++) {
        const int k = k0 + u;
        if (k < n) {
          df d = zcvt(cur[u]) * scale;
          track(dmax, d.hi);
          h = (k == 0) ? d : zw_sub<N1>(d, wprev, h);
          wprev = W(k);
          zput(base + k * P, h);
        }
      }
#pragma unroll
      for (int u = 0; u < ZU; u++) cur[u] = nxt[u];
    }
    df x = df{0.f, 0.f};
    zload_batch<ZU>(cur, base, P, P32, n - 1, -1, n);
    for (int k0 = n - 1; k0 >= 0; k0 -= ZU) {
      if (k0 - ZU >= 0) zload_batch<ZU>(nxt, base, P, P32, k0 - ZU, -1, n);
#pragma unroll
      for (int t = 0; t < ZU; t++) {
        const int k = k0 - t;
        if (k >= 0) {
          const df hk = zcvt(cur[t]);
          x = (k == n - 1) ? zw_mul<N1>(hk, W(k)) : zw_mul<N1>(hk - x, W(k));
          track(umax, x.hi);
          zput(base + k * P, x);
        }
      }
#pragma unroll
      for (int t = 0; t < ZU; t++) cur[t] = nxt[t];
    }
  }
}

// the near -1 form out of line: the few weakly dominant modes of a large grid take a call, and the
// sweeps of all other modes keep the register allocation of the plain form
template <class S, int MODE>
__device__ __noinline__ void z_sweeps_near1(const ZArgs& a, const ZMode& m, S* base, long long P, int n, df scale,
                                            const float2* wt, bool plus1, float& dmax, float& umax) {
  z_sweeps<S, MODE, true>(a, m, base, P, n, scale, wt, plus1, dmax, umax);
}

template <class S, int MODE>
__device__ __forceinline__ void z_line(const ZArgs& a, float& dmax, float& umax) {
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nreal) return;
  // slot s of the (padded) spectral plane -> row, column; padding columns carry no mode
  const unsigned row = a.fd_row.div((unsigned)s);
  const int col = (int)(s - (long long)row * a.row_reals);
  if (col >= a.row_valid) return;
  const long long mi = (long long)row * a.row_modes + (a.cplx ? (col >> 1) : col);
  const ZMode& m = a.modes[mi];
  S* base = reinterpret_cast<S*>(a.data) + s;
  const long long P = a.plane;
  const int n = a.nz;
  const df scale = df{a.scale[0], a.scale[1]};
  const float2* wt = a.wtab + m.woff;
  const int flags = m.flags;
  if (a.only_singular && !(flags & ZF_SINGULAR)) return;
  if (flags & ZF_SINGULAR) {
    z_singular<S>(base, P, n, scale, wt, dmax, umax);
    return;
  }
  // a warp runs the near -1 form when any of its modes needs it (the others convert their w): no
  // warp runs both forms one after the other
  const bool mine = (flags & ZF_NEAR1) != 0;
  if (__any_sync(__activemask(), mine)) z_sweeps_near1<S, MODE>(a, m, base, P, n, scale, wt, !mine, dmax, umax);
  else z_sweeps<S, MODE, false>(a, m, base, P, n, scale, wt, false, dmax, umax);
}

// Checkpointed sweeps of the double-float spill (FP64-class plans).  The forward sweep leaves the
// right-hand sides in place and stores the eliminated value only at the end of each batch of ZU
// planes, in the plan's other spectral buffer (unused while the z stage runs); the back
// substitution re-reads a batch's right-hand sides, recomputes its eliminated values from the
// previous batch's checkpoint (in registers, over the raw values it just loaded) and substitutes.
// HBM traffic per value: 3 + 2/ZU spill values instead of the two-sweep kernel's 4; the recomputed
// forward step is cheap beside the bandwidth it saves (the double-float sweeps are bound by HBM).
// Same arithmetic, in the same order, as the two-sweep kernel.
template <int MODE, bool N1>
__device__ __forceinline__ void z_sweeps_ck(const ZArgs& a, const ZMode& m, float2* base, float2* ck, long long P,
                                            long long CP, int n, df scale, const float2* wt, bool plus1,
                                            float& dmax, float& umax) {
  using S = float2;
  // plus1: this mode stores w itself but runs the near -1 form beside a mode of its warp that needs
  // it; its multipliers are converted to 1 + w on the fly (exact enough away from -1)
  const df one = df{1.f, 0.f};
  df winf = f2df(m.winf), wlast = f2df(m.wlast);
  if (N1 && plus1) { winf = winf + one; wlast = wlast + one; }
  const int wlen = m.wlen;
  auto W = [&](int k) -> df {
    if (k == n - 1) return wlast;
    if (k < wlen) {
      df x = f2df(__ldg(wt + k));
      if (N1 && plus1) x = x + one;
      return x;
    }
    return winf;
  };
  constexpr int ZU = ZBatch<S>::v;
  const int nb = (n + ZU - 1) / ZU;
  S cur[ZU], nxt[ZU];

  if constexpr (MODE != 2) {
    constexpr bool periodic = (MODE == 1);
    const float2* qt = a.qtab + m.qoff;
    const int qlen = periodic ? m.qlen : 0;
    // forward elimination g_k = (s d_k - g_{k-1}) w_k; periodic: y0 = sum q_k s d_k
    df g = df{0.f, 0.f};
    df y0 = df{0.f, 0.f};
    zload<ZU>(cur, base, P, 0, 1, n);
    for (int j = 0; j < nb; j++) {
      const int k0 = j * ZU;
      if (j + 1 < nb) zload<ZU>(nxt, base, P, k0 + ZU, 1, n);
      if (k0 >= wlen && k0 >= qlen && k0 + ZU < n) {
#pragma unroll
        for (int u = 0; u < ZU; u++) {
          const df d = zcvt(cur[u]) * scale;
          track(dmax, d.hi);
          g = zw_mul<N1>(d - g, winf);
        }
      } else {
#pragma unroll
        for (int u = 0; u < ZU; u++) {
          const int k = k0 + u;
          if (k < n) {
            const df d = zcvt(cur[u]) * scale;
            track(dmax, d.hi);
            g = zw_mul<N1>(d - g, W(k));
            if (periodic && k < qlen) y0 = y0 + f2df(__ldg(qt + k)) * d;
          }
        }
      }
      ck[j * CP] = make_float2(g.hi, g.lo);  // g at the last row of batch j
#pragma unroll
      for (int u = 0; u < ZU; u++) cur[u] = nxt[u];
    }
    df c = df{0.f, 0.f}, cg = df{0.f, 0.f};
    if (periodic) {
      c = (y0 + g * f2df(m.igam)) * f2df(m.dsm);  // g == y_{n-1}
      cg = c * f2df(m.gam);
    }
    // back substitution u_k = g_k - w_k u_{k+1} (periodic: v_k), batch by batch from the top
    df u = df{0.f, 0.f};
    zload<ZU>(cur, base, P, (nb - 1) * ZU, 1, n);
    for (int j = nb - 1; j >= 0; j--) {
      const int k0 = j * ZU;
      if (j > 0) zload<ZU>(nxt, base, P, k0 - ZU, 1, n);
      df gk = (j == 0) ? df{0.f, 0.f} : f2df(ck[(j - 1) * CP]);
      const bool fast = k0 >= wlen && k0 >= qlen && k0 + ZU < n;
      if (fast) {
#pragma unroll
        for (int t = 0; t < ZU; t++) {
          gk = zw_mul<N1>(zcvt(cur[t]) * scale - gk, winf);
          cur[t] = make_float2(gk.hi, gk.lo);
        }
#pragma unroll
        for (int t = ZU - 1; t >= 0; t--) {
          u = zw_sub<N1>(zcvt(cur[t]), winf, u);
          track(umax, u.hi);
          zput(base + (k0 + t) * P, u);
        }
      } else {
#pragma unroll
        for (int t = 0; t < ZU; t++) {
          const int k = k0 + t;
          if (k < n) {
            gk = zw_mul<N1>(zcvt(cur[t]) * scale - gk, W(k));
            cur[t] = make_float2(gk.hi, gk.lo);
          }
        }
#pragma unroll
        for (int t = ZU - 1; t >= 0; t--) {
          const int k = k0 + t;
          if (k < n) {
            const df gv = zcvt(cur[t]);
            if (k == n - 1) u = periodic ? zw_sub<N1>(gv, wlast, c) : gv;
            else u = zw_sub<N1>(gv, W(k), u);
            df outv = u;
            if (periodic && k < qlen) outv = u - cg * f2df(__ldg(qt + k));
            track(umax, outv.hi);
            zput(base + k * P, outv);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < ZU; t++) cur[t] = nxt[t];
    }
  } else {
    // transposed factorisation: h_k = s d_k - w_{k-1} h_{k-1},  x_k = (h_k - x_{k+1}) w_k
    df h = df{0.f, 0.f};
    df wprev = df{0.f, 0.f};
    zload<ZU>(cur, base, P, 0, 1, n);
    for (int j = 0; j < nb; j++) {
      const int k0 = j * ZU;
      if (j + 1 < nb) zload<ZU>(nxt, base, P, k0 + ZU, 1, n);
#pragma unroll
      for (int u = 0; u < ZU; u++) {
        const int k = k0 + u;
        if (k < n) {
          const df d = zcvt(cur[u]) * scale;
          track(dmax, d.hi);
          h = (k == 0) ? d : zw_sub<N1>(d, wprev, h);
          wprev = W(k);
        }
      }
      ck[j * CP] = make_float2(h.hi, h.lo);
#pragma unroll
      for (int u = 0; u < ZU; u++) cur[u] = nxt[u];
    }
    df x = df{0.f, 0.f};
    zload<ZU>(cur, base, P, (nb - 1) * ZU, 1, n);
    for (int j = nb - 1; j >= 0; j--) {
      const int k0 = j * ZU;
      if (j > 0) zload<ZU>(nxt, base, P, k0 - ZU, 1, n);
      df hk = (j == 0) ? df{0.f, 0.f} : f2df(ck[(j - 1) * CP]);
      df wp = (k0 == 0) ? df{0.f, 0.f} : W(k0 - 1);
#pragma unroll
      for (int t = 0; t < ZU; t++) {
        const int k = k0 + t;
        if (k < n) {
          const df d = zcvt(cur[t]) * scale;
          hk = (k == 0) ? d : zw_sub<N1>(d, wp, hk);
          wp = W(k);
          cur[t] = make_float2(hk.hi, hk.lo);
        }
      }
#pragma unroll
      for (int t = ZU - 1; t >= 0; t--) {
        const int k = k0 + t;
        if (k < n) {
          const df hv = zcvt(cur[t]);
          x = (k == n - 1) ? zw_mul<N1>(hv, W(k)) : zw_mul<N1>(hv - x, W(k));
          track(umax, x.hi);
          zput(base + k * P, x);
        }
      }
#pragma unroll
      for (int t = 0; t < ZU; t++) cur[t] = nxt[t];
    }
  }
}

template <int MODE>
__device__ __noinline__ void z_sweeps_ck_near1(const ZArgs& a, const ZMode& m, float2* base, float2* ck, long long P,
                                               long long CP, int n, df scale, const float2* wt, bool plus1,
                                               float& dmax, float& umax) {
  z_sweeps_ck<MODE, true>(a, m, base, ck, P, CP, n, scale, wt, plus1, dmax, umax);
}

template <int MODE>
__device__ __forceinline__ void z_line_ck(const ZArgs& a, float& dmax, float& umax) {
  using S = float2;
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nreal) return;
  const unsigned row = a.fd_row.div((unsigned)s);
  const int col = (int)(s - (long long)row * a.row_reals);
  if (col >= a.row_valid) return;
  const long long mi = (long long)row * a.row_modes + (a.cplx ? (col >> 1) : col);
  const ZMode& m = a.modes[mi];
  S* base = reinterpret_cast<S*>(a.data) + s;
  S* ck = reinterpret_cast<S*>(a.ck) + s;
  const long long P = a.plane, CP = a.nreal;
  const int n = a.nz;
  const df scale = df{a.scale[0], a.scale[1]};
  const float2* wt = a.wtab + m.woff;
  if (a.only_singular && !(m.flags & ZF_SINGULAR)) return;
  if (m.flags & ZF_SINGULAR) {
    z_singular<S>(base, P, n, scale, wt, dmax, umax);
    return;
  }
  const bool mine = (m.flags & ZF_NEAR1) != 0;
  if (__any_sync(__activemask(), mine))
    z_sweeps_ck_near1<MODE>(a, m, base, ck, P, CP, n, scale, wt, !mine, dmax, umax);
  else z_sweeps_ck<MODE, false>(a, m, base, ck, P, CP, n, scale, wt, false, dmax, umax);
}

// 4 CTAs of 256 threads per SM (64 registers; the Thomas sweeps spill 56 bytes and run faster than
// at 3 CTAs without spills, measured), 3 for the cyclic sweeps (they would spill 300 bytes at 64)
template <int MODE> struct ZCkMinBlocks { static constexpr int v = (MODE == 1) ? 3 : 4; };

template <int MODE>
__global__ void __launch_bounds__(256, (ZCkMinBlocks<MODE>::v)) k_zsolve_ck(const ZArgs a) {
  float dmax = 0.0f, umax = 0.0f;
  z_line_ck<MODE>(a, dmax, umax);
  range_report(a.rstat, a.dmin, a.umax, gridDim.x, dmax, umax);
}

template <class S, int MODE>
__global__ void __launch_bounds__(256, (ZMinBlocks<S, MODE>::v)) k_zsolve(const ZArgs a) {
  float dmax = 0.0f, umax = 0.0f;
  z_line<S, MODE>(a, dmax, umax);
  range_report(a.rstat, a.dmin, a.umax, gridDim.x, dmax, umax);
}

template <class S>
static cudaError_t launch_z(const ZArgs& a, int mode, unsigned grid, int threads, cudaStream_t st) {
  if (mode == 1) k_zsolve<S, 1><<<grid, threads, 0, st>>>(a);
  else if (mode == 2) k_zsolve<S, 2><<<grid, threads, 0, st>>>(a);
  else k_zsolve<S, 0><<<grid, threads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_zsolve_impl(const ZArgs& a, bool df_spill, bool zper, cudaStream_t st) {
  // the singular mode alone: it is mode (0, 0), real slot 0 (and 1 for a complex mode)
  const int threads = a.only_singular ? 32 : 256;
  const long long grid = a.only_singular ? 1 : (a.nreal + threads - 1) / threads;
  // periodic z is self-adjoint in this factorisation; the transposed sweep is for Thomas only
  const int mode = zper ? 1 : (a.transpose ? 2 : 0);
  if (df_spill) {
    // the double-float spill always runs the checkpointed sweeps (they need the checkpoint buffer)
    if (!a.ck) return cudaErrorInvalidValue;
    if (mode == 1) k_zsolve_ck<1><<<(unsigned)grid, threads, 0, st>>>(a);
    else if (mode == 2) k_zsolve_ck<2><<<(unsigned)grid, threads, 0, st>>>(a);
    else k_zsolve_ck<0><<<(unsigned)grid, threads, 0, st>>>(a);
    return cudaGetLastError();
  }
  return launch_z<float>(a, mode, (unsigned)grid, threads, st);
}

}  // namespace pp
