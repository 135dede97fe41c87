// pp_fft.cuh -- shared-memory mixed-radix (2,3,4,5,7,8) Stockham FFT for a batch of lines.
//
// The complex DFT Y_k = sum_n z_n exp(-2 pi i n k / M) (Sec. "Periodic Boundary Condition")
// of every line of a CTA is computed in place in shared memory by the Stockham
// autosort recursion: with current length n = M/s and radix r (m = n/r), stage
// butterfly (p, q), p < m, q < s, reads z[q + s(p + u m)], u < r, applies an r-point
// DFT and the twiddle exp(-2 pi i p t / n) = w_M^(p t s), and writes y[q + s(r p + t)].
// After the last stage the result is in natural order.  Each thread holds all of its
// butterflies of a stage in registers between two barriers, so the stage can be done in
// place; the host sizes the batch so that a stage never needs more than NB(r)
// butterflies per thread.
#pragma once
#include <type_traits>

#include "pp_arith.cuh"

namespace pp {

constexpr int kMaxStages = 16;

// Shared-memory position of element i of a line: one padding slot after every 32 elements, so
// the strided writes of the early Stockham stages (stride radix x 8..16 bytes) hit distinct banks.
__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

// Unsigned division by a run-time invariant divisor with one multiply-high and two shifts
// (Granlund & Montgomery, "Division by invariant integers using multiplication", 1994):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> min(l,1))) >> max(l-1,0)
// with t = mulhi(m, n); exact for all 32-bit n.
struct FastDiv {
  unsigned d, m, s1, s2;
  static FastDiv make(unsigned dv) {
    FastDiv f;
    unsigned l = 0;
    while ((1ull << l) < dv) l++;
    f.d = dv;
    f.m = (unsigned)((((1ull << 32) * ((1ull << l) - dv)) / dv) + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
  }
  __device__ __forceinline__ unsigned div(unsigned n) const {
    unsigned t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

// butterflies per thread per stage
template <int RAD> struct NBut;
template <> struct NBut<2> { static constexpr int v = 4; };
template <> struct NBut<3> { static constexpr int v = 2; };
template <> struct NBut<4> { static constexpr int v = 2; };
template <> struct NBut<5> { static constexpr int v = 1; };
template <> struct NBut<7> { static constexpr int v = 1; };
template <> struct NBut<8> { static constexpr int v = 1; };
// complex values a thread holds per stage: 8 for radix 2/4/8, 6 / 5 / 7 for radix 3 / 5 / 7 (few
// enough registers for the double-float butterflies).  A launch of a run-time-length kernel is
// valid only if lines_per_cta * M <= (the smallest of these over the line's stages) * threads
// (checked on the host before every launch): then no stage has more butterflies than NB * threads.
__host__ __device__ constexpr int stage_capacity(int rad) {
  return rad == 2 ? 8 : rad == 3 ? 6 : rad == 4 ? 8 : rad == 5 ? 5 : rad == 7 ? 7 : 8;
}
constexpr int kCapPerThread = 8;

// Compile-time lengths transform every line with its own team of MC/VPT consecutive threads, VPT
// (8 or 16) complex values per thread per stage.  Teams of up to one warp synchronise their stages
// with the warp alone; wider teams use the CTA barrier.  The 512-point y kernels, and the FP32 x
// kernels of that length, use VPT = 16 (one warp per line; measured faster), the others VPT = 8.
// Lengths 3 x 2^k (radix-3 last stage) spread the butterflies of all lines over the CTA instead,
// NBut per thread: at most 6 values (two radix-3 butterflies).
constexpr bool ct_pow2(int MC) { return (MC & (MC - 1)) == 0; }
constexpr int ct_values_per_thread(int MC, bool y_lines, bool df_arith) {
  return !ct_pow2(MC) ? 6 : ((MC == 512 && (y_lines || !df_arith)) ? 16 : 8);
}
template <int TPL> __device__ __forceinline__ void team_sync() {
  if constexpr (TPL <= 32) __syncwarp();
  else __syncthreads();
}

// r-point DFTs in registers (forward kernel exp(-2 pi i/r); INV uses the conjugate).
template <class R, bool INV> __device__ __forceinline__ void dft2(cx<R>* a) {
  cx<R> t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}
template <class R, bool INV> __device__ __forceinline__ void dft4(cx<R>* a) {
  cx<R> t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  cx<R> t2 = cadd(a[1], a[3]), t3 = cmul_mi<R, INV>(csub(a[1], a[3]));
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = cadd(t1, t3);
  a[3] = csub(t1, t3);
}
template <class R, bool INV> __device__ __forceinline__ void dft3(cx<R>* a) {
  cx<R> t1 = cadd(a[1], a[2]);
  cx<R> d = csub(a[1], a[2]);
  // t2 = (a1 - a2) * (-+ i sqrt(3)/2)
  cx<R> t2 = cmul_mi<R, INV>(cscale(d, Ar<R>::sqrt3_2()));
  cx<R> m = csub(a[0], chalf(t1));
  a[0] = cadd(a[0], t1);
  a[1] = cadd(m, t2);
  a[2] = csub(m, t2);
}
template <class R, bool INV> __device__ __forceinline__ void dft8(cx<R>* a) {
  cx<R> e[4] = {a[0], a[2], a[4], a[6]};
  cx<R> o[4] = {a[1], a[3], a[5], a[7]};
  dft4<R, INV>(e);
  dft4<R, INV>(o);
  // o1 *= w8, o2 *= w8^2 = -+i, o3 *= w8^3 ; w8 = exp(-+ i pi/4) = (1 -+ i)/sqrt2
  const R s = Ar<R>::sqrt1_2();
  {
    cx<R> v = o[1];
    // (re + im*i)(1 - i)/sqrt2 = ((re + im) + (im - re) i)/sqrt2   [forward]
    // (re + im*i)(1 + i)/sqrt2 = ((re - im) + (im + re) i)/sqrt2   [inverse]
    cx<R> w = INV ? cx<R>{Ar<R>::sub(v.re, v.im), Ar<R>::add(v.im, v.re)}
                  : cx<R>{Ar<R>::add(v.re, v.im), Ar<R>::sub(v.im, v.re)};
    o[1] = cscale(w, s);
  }
  o[2] = cmul_mi<R, INV>(o[2]);
  {
    cx<R> v = o[3];
    // w8^3 = (-1 - i)/sqrt2 [fwd]: (re + im i)(-1 - i) = (-re + im) + (-im - re) i
    // conj: (-1 + i)/sqrt2 [inv]: (re + im i)(-1 + i) = (-re - im) + (re - im) i
    cx<R> w = INV ? cx<R>{Ar<R>::neg(Ar<R>::add(v.re, v.im)), Ar<R>::sub(v.re, v.im)}
                  : cx<R>{Ar<R>::sub(v.im, v.re), Ar<R>::neg(Ar<R>::add(v.im, v.re))};
    o[3] = cscale(w, s);
  }
#pragma unroll
  for (int k = 0; k < 4; k++) {
    a[k] = cadd(e[k], o[k]);
    a[k + 4] = csub(e[k], o[k]);
  }
}

// A constant of the arithmetic type from its FP32 split hi + lo (FP32 keeps hi, the nearest float).
template <class R> __device__ __forceinline__ R kconst(float hi, float lo);
template <> __device__ __forceinline__ float kconst<float>(float hi, float) { return hi; }
template <> __device__ __forceinline__ df kconst<df>(float hi, float lo) { return df{hi, lo}; }

// 5-point DFT.  With t1 = a1 + a4, t2 = a2 + a3, t3 = a1 - a4, t4 = a2 - a3 and c_k, s_k =
// cos, sin(2 pi k / 5):  Y_1, Y_4 = a0 + c1 t1 + c2 t2 -+ i (s1 t3 + s2 t4),
// Y_2, Y_3 = a0 + c2 t1 + c1 t2 -+ i (s2 t3 - s1 t4);  the inverse takes the other sign of i.
template <class R, bool INV> __device__ __forceinline__ void dft5(cx<R>* a) {
  const R c1 = kconst<R>(0x1.3c6ef4p-2f, -0x1.1a02d6p-27f), c2 = kconst<R>(-0x1.9e377ap-1f, 0x1.1a02d6p-27f);
  const R s1 = kconst<R>(0x1.e6f0e2p-1f, -0x1.977560p-26f), s2 = kconst<R>(0x1.2cf230p-1f, 0x1.1d5698p-27f);
  const cx<R> t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]), t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
  const cx<R> A1 = cadd(a[0], cadd(cscale(t1, c1), cscale(t2, c2)));
  const cx<R> A2 = cadd(a[0], cadd(cscale(t1, c2), cscale(t2, c1)));
  const cx<R> B1 = cmul_mi<R, INV>(cadd(cscale(t3, s1), cscale(t4, s2)));
  const cx<R> B2 = cmul_mi<R, INV>(csub(cscale(t3, s2), cscale(t4, s1)));
  a[0] = cadd(a[0], cadd(t1, t2));
  a[1] = cadd(A1, B1);
  a[4] = csub(A1, B1);
  a[2] = cadd(A2, B2);
  a[3] = csub(A2, B2);
}

// 7-point DFT.  With t_m = a_m + a_{7-m}, u_m = a_m - a_{7-m} (m = 1..3) and c_j, s_j =
// cos, sin(2 pi j / 7):  Y_k, Y_{7-k} = a0 + sum_m cos(2 pi k m/7) t_m -+ i sum_m sin(2 pi k m/7) u_m,
// k = 1..3 (cos(2 pi k m/7) = c_{km mod 7}, c_{7-j} = c_j, s_{7-j} = -s_j).
template <class R, bool INV> __device__ __forceinline__ void dft7(cx<R>* a) {
  const R c1 = kconst<R>(0x1.3f3a0ep-1f, 0x1.45f6e8p-28f), c2 = kconst<R>(-0x1.c7b90ep-3f, -0x1.8122c0p-30f);
  const R c3 = kconst<R>(-0x1.cd4bcap-1f, -0x1.396b8ep-26f), s1 = kconst<R>(0x1.904c38p-1f, -0x1.5f4436p-26f);
  const R s2 = kconst<R>(0x1.f329c0p-1f, 0x1.563a5ap-27f), s3 = kconst<R>(0x1.bc4c04p-2f, 0x1.ae3578p-27f);
  const cx<R> t1 = cadd(a[1], a[6]), t2 = cadd(a[2], a[5]), t3 = cadd(a[3], a[4]);
  const cx<R> u1 = csub(a[1], a[6]), u2 = csub(a[2], a[5]), u3 = csub(a[3], a[4]);
  const cx<R> A1 = cadd(a[0], cadd(cadd(cscale(t1, c1), cscale(t2, c2)), cscale(t3, c3)));
  const cx<R> A2 = cadd(a[0], cadd(cadd(cscale(t1, c2), cscale(t2, c3)), cscale(t3, c1)));
  const cx<R> A3 = cadd(a[0], cadd(cadd(cscale(t1, c3), cscale(t2, c1)), cscale(t3, c2)));
  const cx<R> B1 = cmul_mi<R, INV>(cadd(cadd(cscale(u1, s1), cscale(u2, s2)), cscale(u3, s3)));
  const cx<R> B2 = cmul_mi<R, INV>(csub(csub(cscale(u1, s2), cscale(u2, s3)), cscale(u3, s1)));
  const cx<R> B3 = cmul_mi<R, INV>(cadd(csub(cscale(u1, s3), cscale(u2, s1)), cscale(u3, s2)));
  a[0] = cadd(a[0], cadd(cadd(t1, t2), t3));
  a[1] = cadd(A1, B1);
  a[6] = csub(A1, B1);
  a[2] = cadd(A2, B2);
  a[5] = csub(A2, B2);
  a[3] = cadd(A3, B3);
  a[4] = csub(A3, B3);
}

template <class R, int RAD, bool INV> __device__ __forceinline__ void dft_r(cx<R>* a) {
  if constexpr (RAD == 2) dft2<R, INV>(a);
  else if constexpr (RAD == 3) dft3<R, INV>(a);
  else if constexpr (RAD == 4) dft4<R, INV>(a);
  else if constexpr (RAD == 5) dft5<R, INV>(a);
  else if constexpr (RAD == 7) dft7<R, INV>(a);
  else dft8<R, INV>(a);
}

// One Stockham stage over all lines of the CTA.  buf: lines of M complex at stride ldm.
// tw: w_M^j = exp(-2 pi i j / M), j < M (shared memory).
template <class R, int RAD, bool INV>
__device__ __forceinline__ void fft_stage(cx<R>* buf, int nlines, int ldm, int s, const FastDiv& fd_nbl,
                                          const FastDiv& fd_s, const cx<R>* tw) {
  constexpr int NB = NBut<RAD>::v;
  const int nbl = (int)fd_nbl.d;
  const int total = nlines * nbl;
  cx<R> a[NB][RAD];
  int lj[NB];  // butterfly -> (line, j), computed once
#pragma unroll
  for (int i = 0; i < NB; i++) {
    int b = threadIdx.x + i * blockDim.x;
    lj[i] = -1;
    if (b < total) {
      int line = (int)fd_nbl.div((unsigned)b), j = b - line * nbl;
      lj[i] = line * ldm + j;
      const cx<R>* x = buf + line * ldm;
#pragma unroll
      for (int u = 0; u < RAD; u++) a[i][u] = x[pad(j + u * nbl)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; i++) {
    if (lj[i] >= 0) {
      int b = threadIdx.x + i * blockDim.x;
      int line = (int)fd_nbl.div((unsigned)b), j = b - line * nbl;
      int p = (int)fd_s.div((unsigned)j), q = j - p * s;
      dft_r<R, RAD, INV>(a[i]);
      cx<R>* y = buf + line * ldm;
      const int o = q + s * RAD * p;
      y[pad(o)] = a[i][0];
      const int ps = p * s;
      if (s == nbl) {
        // last stage: p = 0, every twiddle is 1
#pragma unroll
        for (int t = 1; t < RAD; t++) y[pad(o + s * t)] = a[i][t];
      } else {
#pragma unroll
        for (int t = 1; t < RAD; t++) {
          cx<R> w = tw[ps * t];
          y[pad(o + s * t)] = INV ? cmulc(a[i][t], w) : cmul(a[i][t], w);
        }
      }
    }
  }
  __syncthreads();
}

struct FftPlan {
  int M;              // complex length
  int nst;            // number of stages
  int rad[kMaxStages];
  FastDiv nbl[kMaxStages];  // M / rad per stage
  FastDiv s[kMaxStages];    // product of the earlier radices
};

// All stages of a run-time length.  R57: the kernel also carries the radix-5 and radix-7
// butterflies (their registers would otherwise weigh on every 2^a 3^b length).
template <class R, bool INV, bool R57>
__device__ __forceinline__ void fft_lines(cx<R>* buf, int nlines, int ldm, const FftPlan& fp, const cx<R>* tw) {
  int s = 1;
  for (int st = 0; st < fp.nst; st++) {
    int r = fp.rad[st];
    if (r == 8) fft_stage<R, 8, INV>(buf, nlines, ldm, s, fp.nbl[st], fp.s[st], tw);
    else if (r == 4) fft_stage<R, 4, INV>(buf, nlines, ldm, s, fp.nbl[st], fp.s[st], tw);
    else if (r == 3) fft_stage<R, 3, INV>(buf, nlines, ldm, s, fp.nbl[st], fp.s[st], tw);
    else if (R57 && r == 5) fft_stage<R, (R57 ? 5 : 2), INV>(buf, nlines, ldm, s, fp.nbl[st], fp.s[st], tw);
    else if (R57 && r == 7) fft_stage<R, (R57 ? 7 : 2), INV>(buf, nlines, ldm, s, fp.nbl[st], fp.s[st], tw);
    else fft_stage<R, 2, INV>(buf, nlines, ldm, s, fp.nbl[st], fp.s[st], tw);
    s *= r;
  }
}

// ---------------------------------------------------------------- compile-time length
// For a length MC known at compile time (a power of two, or 3 x 2^k) the stage sequence (radix 8
// while it divides, then 4, then 2, then 3) and every index division are resolved by the compiler.
//
// Addressing: with powers of two, pad(j + u nbl) = pad(j) + u nbl + (u nbl >> 5) and, for the
// output position o = q + S r p (q < S), pad(o + S t) = pad(o) + S t + (S t >> 5), so every
// shared-memory access of a butterfly is one base address plus a compile-time offset (3 x 2^k
// lengths compute each padded index).
// Twiddles are stored per stage in butterfly order: stage k (stride S, radix r, p < MC/(S r))
// keeps w_MC^(p S t), t = 1..r-1, at off_k + p (r-1) + t-1; off_k = MC - MC/S (the sizes
// telescope), and the last stage (p = 0, all twiddles 1) keeps none.
template <int REM> struct CtRadix {
  static constexpr int v = (REM % 8 == 0) ? 8 : (REM % 4 == 0) ? 4 : (REM % 2 == 0) ? 2 : 3;
};

template <class R, int RAD, bool INV, int MC, int VPT, int S, int TWOFF>
__device__ __forceinline__ void fft_stage_ct(cx<R>* buf, int nlines, int ldm, const cx<R>* tw) {
  constexpr int nbl = MC / RAD;
  if constexpr (!ct_pow2(MC)) {
    // 3 x 2^k: the butterflies of all lines spread over the CTA, CTA barriers
    constexpr int NB = NBut<RAD>::v;
    const int total = nlines * nbl;
    cx<R> a[NB][RAD];
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const int b = threadIdx.x + i * blockDim.x;
      if (b < total) {
        const cx<R>* x = buf + (b / nbl) * ldm;
        const int j = b % nbl;
#pragma unroll
        for (int u = 0; u < RAD; u++) a[i][u] = x[pad(j + u * nbl)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const int b = threadIdx.x + i * blockDim.x;
      if (b < total) {
        const int j = b % nbl;
        const int p = j / S, q = j % S;
        dft_r<R, RAD, INV>(a[i]);
        cx<R>* y = buf + (b / nbl) * ldm;
        const int o = q + S * RAD * p;
        y[pad(o)] = a[i][0];
        if constexpr (S * RAD == MC) {
#pragma unroll
          for (int t = 1; t < RAD; t++) y[pad(o + S * t)] = a[i][t];
        } else {
          const cx<R>* w = tw + TWOFF + p * (RAD - 1);
#pragma unroll
          for (int t = 1; t < RAD; t++) y[pad(o + S * t)] = INV ? cmulc(a[i][t], w[t - 1]) : cmul(a[i][t], w[t - 1]);
        }
      }
    }
    __syncthreads();
  } else {
    constexpr int TPL = MC / VPT;
    constexpr int NB = nbl / TPL;  // butterflies per thread
    static_assert(NB * TPL == nbl && NB * RAD <= 16, "team covers the line");
    // FP32 lines of 512 points (radix 8, 8, 8): the first stage writes its output transposed, as an
    // 8 x 64 array (output 8p + t at 64t + p), and the second stage reads it so.  The first stage's
    // stores are then consecutive across a warp instead of 64 bytes apart (a two-way bank conflict
    // on every one of its 8-byte stores), and with the one-in-32 padding the second stage's loads
    // stay conflict-free and at compile-time offsets: pad(64a + b + 8u) = 66a + b + 8u + (8u >> 5)
    // for a = j mod 8, b = j / 8 < 8.
    constexpr bool TR_OUT = std::is_same<R, float>::value && MC == 512 && RAD == 8 && S == 1;
    constexpr bool TR_IN = std::is_same<R, float>::value && MC == 512 && RAD == 8 && S == 8;
    const int line = (int)threadIdx.x / TPL, lt = (int)threadIdx.x % TPL;
    const bool act = line < nlines;
    cx<R> a[NB][RAD];
    if (act) {
#pragma unroll
      for (int i = 0; i < NB; i++) {
        if constexpr (TR_IN) {
          const int j = lt + i * TPL;
          const cx<R>* x = buf + line * ldm + 66 * (j & 7) + (j >> 3);
#pragma unroll
          for (int u = 0; u < RAD; u++) a[i][u] = x[8 * u + ((8 * u) >> 5)];
        } else {
          const cx<R>* x = buf + line * ldm + pad(lt + i * TPL);
#pragma unroll
          for (int u = 0; u < RAD; u++) a[i][u] = x[u * nbl + ((u * nbl) >> 5)];
        }
      }
    }
    team_sync<TPL>();
#pragma unroll
    for (int i = 0; i < NB; i++) {
      if (act) {
        const int j = lt + i * TPL;
        const int p = j / S, q = j % S;
        dft_r<R, RAD, INV>(a[i]);
        if constexpr (TR_OUT) {
          // output 8p + t at pad(64t + p) = pad(p) + 66t (p < 64)
          cx<R>* y = buf + line * ldm + pad(p);
          const cx<R>* w = tw + TWOFF + p * (RAD - 1);
          y[0] = a[i][0];
#pragma unroll
          for (int t = 1; t < RAD; t++) y[66 * t] = INV ? cmulc(a[i][t], w[t - 1]) : cmul(a[i][t], w[t - 1]);
          continue;
        }
        cx<R>* y = buf + line * ldm + pad(q + S * RAD * p);
        y[0] = a[i][0];
        if constexpr (S * RAD == MC) {
          // last stage: p = 0, every twiddle is 1
#pragma unroll
          for (int t = 1; t < RAD; t++) y[S * t + ((S * t) >> 5)] = a[i][t];
        } else {
          const cx<R>* w = tw + TWOFF + p * (RAD - 1);  // w[t-1] = w_MC^(p S t)
#pragma unroll
          for (int t = 1; t < RAD; t++)
            y[S * t + ((S * t) >> 5)] = INV ? cmulc(a[i][t], w[t - 1]) : cmul(a[i][t], w[t - 1]);
        }
      }
    }
    team_sync<TPL>();
  }
}

// tw: the per-stage table of load_stage_twiddles
template <class R, bool INV, int MC, int VPT, int S = 1, int TWOFF = 0>
__device__ __forceinline__ void fft_lines_ct(cx<R>* buf, int nlines, int ldm, const cx<R>* tw) {
  if constexpr (S < MC) {
    constexpr int RAD = CtRadix<MC / S>::v;
    fft_stage_ct<R, RAD, INV, MC, VPT, S, TWOFF>(buf, nlines, ldm, tw);
    constexpr int NEXT = (S * RAD < MC) ? TWOFF + (MC / (S * RAD)) * (RAD - 1) : TWOFF;
    fft_lines_ct<R, INV, MC, VPT, S * RAD, NEXT>(buf, nlines, ldm, tw);
  }
}

// Radix-8 stage with the stride S = 2^lgS known only at run time (line teams as above).  The
// double-float butterfly is long (~900 instructions); running all radix-8 stages through one copy
// of it keeps the kernel's hot code within the instruction cache.  Same addressing and twiddle
// table as fft_stage_ct (radix-8 stages come first, so this stage's twiddles start at MC - MC/S).
template <class R, bool INV, int MC, int VPT>
__device__ __forceinline__ void fft_stage8_rt(cx<R>* buf, int nlines, int ldm, const cx<R>* tw, int lgS, bool last) {
  constexpr int nbl = MC / 8;
  constexpr int TPL = MC / VPT;
  constexpr int NB = nbl / TPL;  // butterflies per thread
  const int line = (int)threadIdx.x / TPL, lt = (int)threadIdx.x % TPL;
  const bool act = line < nlines;
  cx<R> a[NB][8];
  if (act) {
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const cx<R>* x = buf + line * ldm + pad(lt + i * TPL);
#pragma unroll
      for (int u = 0; u < 8; u++) a[i][u] = x[u * nbl + ((u * nbl) >> 5)];
    }
  }
  team_sync<TPL>();
#pragma unroll
  for (int i = 0; i < NB; i++) {
    if (act) {
      const int j = lt + i * TPL;
      const int p = j >> lgS, q = j & ((1 << lgS) - 1);
      dft8<R, INV>(a[i]);
      cx<R>* y = buf + line * ldm + pad(q + ((8 * p) << lgS));
      y[0] = a[i][0];
      if (last) {
#pragma unroll
        for (int t = 1; t < 8; t++) y[(t << lgS) + ((t << lgS) >> 5)] = a[i][t];
      } else {
        const cx<R>* w = tw + (MC - (MC >> lgS)) + p * 7;
#pragma unroll
        for (int t = 1; t < 8; t++)
          y[(t << lgS) + ((t << lgS) >> 5)] = INV ? cmulc(a[i][t], w[t - 1]) : cmul(a[i][t], w[t - 1]);
      }
    }
  }
  team_sync<TPL>();
}

// All stages of a power-of-two length: the radix-8 stages in a loop (not unrolled), then the
// remaining radix-4 or radix-2 stage.  Same stage sequence and results as fft_lines_ct.
template <class R, bool INV, int MC, int VPT>
__device__ __forceinline__ void fft_lines_lp(cx<R>* buf, int nlines, int ldm, const cx<R>* tw) {
  constexpr int L8 = (MC >= 8) ? (31 - __builtin_clz(MC)) / 3 : 0;
  constexpr int REM = MC >> (3 * L8);
#pragma unroll 1
  for (int st = 0; st < L8; st++)
    fft_stage8_rt<R, INV, MC, VPT>(buf, nlines, ldm, tw, 3 * st, REM == 1 && st == L8 - 1);
  if constexpr (REM == 4) fft_stage_ct<R, 4, INV, MC, VPT, MC / 4, 0>(buf, nlines, ldm, tw);
  if constexpr (REM == 2) fft_stage_ct<R, 2, INV, MC, VPT, MC / 2, 0>(buf, nlines, ldm, tw);
}

}  // namespace pp
