// pp_lines.cuh -- batched line transforms along x (contiguous lines) and y (strided columns).
//
// Every transform of the paper's table of forward/backward transforms is computed through a
// complex FFT with pre- and post-processing (Sec. "Boundary Conditions": pre-processing,
// complex Fourier transform, post-processing):
//   * real DFT of length N (periodic): the even/odd samples packed as one complex line of
//     length M = N/2, FFT, then the Hermitian split X_k = E_k + w_N^k O_k;
//   * DCT-II ("DCT10", Neumann): Makhoul's reordering (even samples in order, odd samples
//     reversed), a real DFT, and the twiddle exp(-i pi k / 2N), real part; the values of
//     index N-k come from the same complex number (minus its imaginary part);
//   * DST-II ("DST10", Dirichlet): DCT-II of the sign-alternated line, output reversed;
//   * their inverses DCT-III / DST-III ("DCT01"/"DST01") by the reverse steps;
//   * DCT-IV / DST-IV (one Dirichlet and one Neumann face) via a length-N/2 complex FFT with
//     pre-twiddle exp(-i pi (4n+1)/4N) and post-twiddle exp(-i pi k/N).
// All inverse transforms are unnormalised syntheses; the constant inverse weights (1/N, or
// 2/N for type IV) are applied once, in the tridiagonal solve.
//
// One CTA transforms `lpc` lines in shared memory: x lines are `lpc` consecutive rows, y lines
// are `tx` adjacent columns of one plane (times 2 when the real and imaginary parts of complex
// columns are transformed as separate real lines).  Pre-processing reads global memory (x:
// consecutive threads along a line; y: consecutive threads across columns, so every access is
// a coalesced row segment), the FFT runs in place in shared memory, post-processing writes
// global memory in the same patterns.  The kernels are templated on the complex FFT length MC
// (MC = a power of two 8..1024, or 3 x 2^k 24..768: the stage sequence and all index divisions
// are compile-time, and for powers of two each line has its own thread team; MC = 0: the length is read from the plan at run time,
// radices 2, 3, 4, 8; MC = -1: run-time length with radix-5/7 stages as well).
#pragma once
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "pp_internal.h"

namespace pp {

// cp.async copy of one complex value from global to shared memory (16 bytes: bypasses L1;
// 8 bytes: through L1), and the commit / wait of this thread's copies.
template <class R> __device__ __forceinline__ void cp_async_cx(cx<R>* s, const cx<R>* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  const size_t ga = __cvta_generic_to_global(g);
  if constexpr (sizeof(cx<R>) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(ga) : "memory");
  } else {
    static_assert(sizeof(cx<R>) == 8, "complex value of 8 or 16 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(ga) : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// base offsets (in reals) of global line g of the launch
__device__ __forceinline__ long long line_base(const LineArgs& a, unsigned g, bool out) {
  unsigned plane = a.fd_lpp.div(g);
  unsigned r = g - plane * (unsigned)a.lines_per_plane;
  unsigned c = a.fd_parts.div(r), part = r - c * (unsigned)a.parts;
  return out ? (long long)plane * a.out_plane + (long long)c * a.out_line + part
             : (long long)plane * a.in_plane + (long long)c * a.in_line + part;
}

// Visit every (line L, item k) of the tile.  x: k fastest (consecutive threads along a line);
// y: L fastest (consecutive threads across columns).  KC: compile-time item count (0: fdk).
template <bool OY, int KC, class F>
__device__ __forceinline__ void for_items(const LineArgs& a, int nl, const FastDiv& fdk, F&& fn) {
  const int K = KC ? KC : (int)fdk.d;
  const int tot = (OY ? a.lpc : nl) * K;
#pragma unroll 4
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    int L, k;
    if (OY) {
      unsigned q = a.fd_lpc.div((unsigned)t);
      L = t - (int)(q * a.fd_lpc.d);
      k = (int)q;
      if (L >= nl) continue;
    } else {
      if constexpr (KC > 0) {
        L = t / KC;
        k = t % KC;
      } else {
        unsigned q = fdk.div((unsigned)t);
        L = (int)q;
        k = t - (int)q * K;
      }
    }
    fn(L, k);
  }
}

// Vector access to 2 or 4 consecutive reals at a real offset that is a multiple of 2 / 4
// (rows of x tiles are 16-byte aligned; the host checks the array pointers).
// raw(): the loaded bits, cvt(): their conversion to R (split so that a batch of loads can be
// issued before the first conversion waits for its data).
template <class R, class S> struct Vec;
template <> struct Vec<df, double> {
  using raw_t = double2;
  __device__ static __forceinline__ raw_t raw(const double* p, long long o) {
    return __ldg(reinterpret_cast<const double2*>(p + o));
  }
  __device__ static __forceinline__ void cvt(raw_t a, df* v) { v[0] = df_from_double(a.x); v[1] = df_from_double(a.y); }
  __device__ static __forceinline__ void ld2(const double* p, long long o, df* v) { cvt(raw(p, o), v); }
  __device__ static __forceinline__ void st2(double* p, long long o, const df* v) {
    *reinterpret_cast<double2*>(p + o) = make_double2(df_to_double(v[0]), df_to_double(v[1]));
  }
};
template <> struct Vec<df, float2> {
  using raw_t = float4;
  __device__ static __forceinline__ raw_t raw(const float2* p, long long o) {
    return __ldg(reinterpret_cast<const float4*>(p + o));
  }
  __device__ static __forceinline__ void cvt(raw_t a, df* v) { v[0] = df{a.x, a.y}; v[1] = df{a.z, a.w}; }
  __device__ static __forceinline__ void ld2(const float2* p, long long o, df* v) { cvt(raw(p, o), v); }
  __device__ static __forceinline__ void st2(float2* p, long long o, const df* v) {
    *reinterpret_cast<float4*>(p + o) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
  }
};
template <> struct Vec<float, double> {
  using raw_t = double2;
  __device__ static __forceinline__ raw_t raw(const double* p, long long o) {
    return __ldg(reinterpret_cast<const double2*>(p + o));
  }
  __device__ static __forceinline__ void cvt(raw_t a, float* v) { v[0] = f32_from_double(a.x); v[1] = f32_from_double(a.y); }
  __device__ static __forceinline__ void ld2(const double* p, long long o, float* v) { cvt(raw(p, o), v); }
  __device__ static __forceinline__ void st2(double* p, long long o, const float* v) {
    *reinterpret_cast<double2*>(p + o) = make_double2((double)v[0], (double)v[1]);
  }
};
template <> struct Vec<float, float> {
  using raw_t = float2;
  __device__ static __forceinline__ raw_t raw(const float* p, long long o) {
    return __ldg(reinterpret_cast<const float2*>(p + o));
  }
  __device__ static __forceinline__ void cvt(raw_t a, float* v) { v[0] = a.x; v[1] = a.y; }
  __device__ static __forceinline__ void ld2(const float* p, long long o, float* v) { cvt(raw(p, o), v); }
  __device__ static __forceinline__ void st2(float* p, long long o, const float* v) {
    *reinterpret_cast<float2*>(p + o) = make_float2(v[0], v[1]);
  }
};

// 16-byte access to V adjacent reals of a y-tile row (4 FP32 or 2 double-float spill reals).
template <class R, class S> struct VecN;
template <> struct VecN<float, float> {
  static constexpr int V = 4;
  __device__ static __forceinline__ void ld(const float* p, long long o, float* v) {
    float4 a = __ldg(reinterpret_cast<const float4*>(p + o));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  __device__ static __forceinline__ void st(float* p, long long o, const float* v) {
    *reinterpret_cast<float4*>(p + o) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct VecN<df, float2> {
  static constexpr int V = 2;
  __device__ static __forceinline__ void ld(const float2* p, long long o, df* v) {
    float4 a = __ldg(reinterpret_cast<const float4*>(p + o));
    v[0] = df{a.x, a.y}; v[1] = df{a.z, a.w};
  }
  __device__ static __forceinline__ void st(float2* p, long long o, const df* v) {
    *reinterpret_cast<float4*>(p + o) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
  }
};
// nv (<= V) adjacent reals: one vector access for a full group, scalar accesses for a partial one
template <class R, class S> __device__ __forceinline__ void ldn(const S* p, long long o, int nv, R* v) {
  constexpr int V = VecN<R, S>::V;
  if (nv == V) { VecN<R, S>::ld(p, o, v); return; }
#pragma unroll
  for (int i = 0; i < V; i++) v[i] = (i < nv) ? Io<R, S>::ld(p, o + i) : Ar<R>::zero();
}
template <class R, class S> __device__ __forceinline__ void stn(S* p, long long o, int nv, const R* v) {
  constexpr int V = VecN<R, S>::V;
  if (nv == V) { VecN<R, S>::st(p, o, v); return; }
#pragma unroll
  for (int i = 0; i < V; i++)
    if (i < nv) Io<R, S>::st(p, o + i, v[i]);
}

// 16 bytes of VC = 2 adjacent FP32 complex lines of a tile row (complex columns: line L at real
// offset 2L); nv (<= VC) lines of a partial group.
template <class R, class S> struct CVec;
template <> struct CVec<float, float> {
  static constexpr int VC = 2;
  __device__ static __forceinline__ void ld(const float* p, long long o, int nv, cx<float>* z) {
    if (nv == 2) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p + o));
      z[0] = cx<float>{v.x, v.y};
      z[1] = cx<float>{v.z, v.w};
    } else {
      z[0] = cx<float>{p[o], p[o + 1]};
      z[1] = cx<float>{0.0f, 0.0f};
    }
  }
  __device__ static __forceinline__ void st(float* p, long long o, int nv, const cx<float>* z) {
    if (nv == 2) {
      *reinterpret_cast<float4*>(p + o) = make_float4(z[0].re, z[0].im, z[1].re, z[1].im);
    } else {
      p[o] = z[0].re;
      p[o + 1] = z[0].im;
    }
  }
};

// y tiles with contiguous rows: visit (group of V adjacent lines starting at L0, item k); consecutive
// threads take consecutive groups, so a warp's accesses are runs of 16-byte vectors.  nv = lines of
// the group (V, or fewer for the last group of a partial tile).  KC: compile-time item count (0: fdk).
template <int V, int KC, class F>
__device__ __forceinline__ void for_groups(const LineArgs& a, int nl, const FastDiv& fdk, F&& fn) {
  const int K = KC ? KC : (int)fdk.d;
  const int G = (int)a.fd_gpc.d;
  const int tot = G * K;
#pragma unroll 2
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const unsigned q = a.fd_gpc.div((unsigned)t);
    const int L0 = (t - (int)q * G) * V;
    if (L0 >= nl) continue;
    fn(L0, (int)q, min(V, nl - L0));
  }
}

// Batched form of for_items for x tiles of a compile-time length: a thread first issues the loads
// of U items (ld returns their raw bits), then converts and stores them (st), so U items' global
// loads are in flight together; a plain loop waits for each load before the shared-memory store
// that the next load cannot pass.  (Measured: x kernels 4-11% faster; the y tiles' 16-byte loads
// gained nothing, and the FP32 y kernels lost occupancy to the extra registers.)
// Batch size: `full` items for the compile-time power-of-two lengths from 256 on, half of it
// elsewhere (their kernels have fewer registers to spare under the caps; the FP32 kernels' 48
// take half as well).
constexpr int pre_batch(int MC, int full) { return (MC >= 256 && (MC & (MC - 1)) == 0) ? full : (full > 1 ? full / 2 : 1); }

// x tiles of the compile-time power-of-two kernels: when the tile is full and the CTA has one
// team of TPL threads per line, thread k0 of line L takes the items k0 + TPL i (compile-time i);
// KC = M/2 + 1 adds the middle item k = M/2.  XTeam::ok(a, nl) tells whether the tile qualifies.
template <class R, int MC> struct XTeam {
  static constexpr bool ct = MC >= 64 && (MC & (MC - 1)) == 0;
  static constexpr int TPL = ct ? MC / ct_values_per_thread(MC, false, std::is_same<R, df>::value) : 1;
  __device__ static __forceinline__ bool ok(const LineArgs& a, int nl) {
    return ct && nl == a.lpc && (int)blockDim.x == TPL * a.lpc;
  }
};
template <class R, bool OY, int MC, int KC, class F>
__device__ __forceinline__ void for_items_x(const LineArgs& a, int nl, const FastDiv& fdk, F&& fn) {
  if constexpr (!OY && XTeam<R, MC>::ct) {
    constexpr int TPL = XTeam<R, MC>::TPL;
    static_assert(KC == MC || KC == MC / 2 || KC == MC / 2 + 1, "item counts of the x kinds");
    if (XTeam<R, MC>::ok(a, nl)) {
      const int L = (int)threadIdx.x / TPL, k0 = (int)threadIdx.x % TPL;
      constexpr int NF = (KC == MC) ? MC / TPL : MC / 2 / TPL;
#pragma unroll
      for (int i = 0; i < NF; i++) fn(L, k0 + TPL * i);
      if (KC == MC / 2 + 1 && k0 == 0) fn(L, MC / 2);
      return;
    }
  }
  for_items<OY, KC>(a, nl, fdk, fn);
}

template <int KC, int U, class LD, class ST>
__device__ __forceinline__ void for_items_xb(int nl, LD&& ld, ST&& st) {
  const int tot = nl * KC;
  for (int t0 = threadIdx.x; t0 < tot; t0 += U * (int)blockDim.x) {
    decltype(ld(0, 0)) r[U];
    int L[U], k[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int t = t0 + u * (int)blockDim.x;
      L[u] = t < tot ? t / KC : -1;
      k[u] = t % KC;
      if (L[u] >= 0) r[u] = ld(L[u], k[u]);
    }
#pragma unroll
    for (int u = 0; u < U; u++)
      if (L[u] >= 0) st(L[u], k[u], r[u]);
  }
}

// y tiles of the compile-time power-of-two kernels: when the tile is full and the CTA has one
// thread per (group, k0), k0 < KS, every thread takes the items k0 + KS i (compile-time i) of its
// group, with no division and no bounds or partial-group tests; the Hermitian-pair kinds
// (KC = M/2 + 1 items) add the middle item k = M/2.  Other tiles take for_groups.
template <class R, int MC, int V, int KC, class F>
__device__ __forceinline__ void for_groups_y(const LineArgs& a, int nl, const FastDiv& fdk, F&& fn) {
  if constexpr (MC >= 64 && (MC & (MC - 1)) == 0) {
    constexpr int VPT = ct_values_per_thread(MC, true, std::is_same<R, df>::value);
    constexpr int KS = V * (MC / VPT);
    constexpr int NI = MC / KS;
    static_assert(KC == MC || KC == MC / 2 + 1, "item counts of the y kinds");
    static_assert(NI % 2 == 0, "half of a thread's items lie below M/2");
    const int G = a.lpc / V;
    if (nl == a.lpc && (G & (G - 1)) == 0 && (int)blockDim.x == KS * G) {
      const int lg = __ffs(G) - 1;
      const int L0 = ((int)threadIdx.x & (G - 1)) * V;
      const int k0 = (int)threadIdx.x >> lg;
      constexpr int NF = (KC == MC) ? NI : NI / 2;
#pragma unroll
      for (int i = 0; i < NF; i++) fn(L0, k0 + KS * i, V);
      if (KC != MC && k0 == 0) fn(L0, MC / 2, V);
      return;
    }
  }
  for_groups<V, KC>(a, nl, fdk, fn);
}

// for_groups_y with every item's loads issued before any item is converted and stored: the FP32 y
// kernels' forward pre-processing was bound by load latency (1024^3 y-forward 2.49 -> 2.18 ms,
// measured); the inverse kinds and the double-float kernels (bound by issue, capped in registers)
// gained nothing and keep for_groups_y.
template <class R, int MC, int V, int KC, class LD, class ST>
__device__ __forceinline__ void for_groups_yb(const LineArgs& a, int nl, const FastDiv& fdk, LD&& ld, ST&& st) {
  if constexpr (std::is_same<R, float>::value && MC >= 64 && (MC & (MC - 1)) == 0) {
    constexpr int VPT = ct_values_per_thread(MC, true, false);
    constexpr int KS = V * (MC / VPT);
    constexpr int NI = MC / KS;
    static_assert(KC == MC, "full item sets");
    const int G = a.lpc / V;
    if (nl == a.lpc && (G & (G - 1)) == 0 && (int)blockDim.x == KS * G) {
      const int lg = __ffs(G) - 1;
      const int L0 = ((int)threadIdx.x & (G - 1)) * V;
      const int k0 = (int)threadIdx.x >> lg;
      decltype(ld(0, 0, 0)) r[NI];
#pragma unroll
      for (int i = 0; i < NI; i++) r[i] = ld(L0, k0 + KS * i, V);
#pragma unroll
      for (int i = 0; i < NI; i++) st(L0, k0 + KS * i, V, r[i]);
      return;
    }
  }
  for_groups_y<R, MC, V, KC>(a, nl, fdk, [&](int L0, int k, int nv) { st(L0, k, nv, ld(L0, k, nv)); });
}

// for_items_xb with the team mapping of for_items_x where the tile qualifies (U | the item count).
// Used by the forward x kinds; the inverse kinds' loops measured slower with it (larger code in the
// kernel that also converts to FP64).
template <class R, int MC, int KC, int U, class LD, class ST>
__device__ __forceinline__ void for_items_xbt(const LineArgs& a, int nl, LD&& ld, ST&& st) {
  if constexpr (XTeam<R, MC>::ct) {
    constexpr int TPL = XTeam<R, MC>::TPL;
    constexpr int NF = MC / 2 / TPL;
    static_assert(KC == MC / 2 || KC == MC / 2 + 1, "item counts of the batched x kinds");
    static_assert(NF % U == 0, "whole batches");
    if (XTeam<R, MC>::ok(a, nl)) {
      const int L = (int)threadIdx.x / TPL, k0 = (int)threadIdx.x % TPL;
#pragma unroll
      for (int i0 = 0; i0 < NF; i0 += U) {
        decltype(ld(0, 0)) r[U];
#pragma unroll
        for (int u = 0; u < U; u++) r[u] = ld(L, k0 + TPL * (i0 + u));
#pragma unroll
        for (int u = 0; u < U; u++) st(L, k0 + TPL * (i0 + u), r[u]);
      }
      if (KC == MC / 2 + 1 && k0 == 0) st(L, MC / 2, ld(L, MC / 2));
      return;
    }
  }
  for_items_xb<KC, U>(nl, ld, st);
}

template <class R, class SI> struct SrcGlobal {
  using elem_t = SI;
  const SI* in;
  const long long* bases;  // per-line bases (shared memory)
  long long pos;           // stride between positions of a line
  __device__ __forceinline__ long long base(int L) const { return bases[L]; }
  __device__ __forceinline__ R ld(long long b, int j) const { return Io<R, SI>::ld(in, b + (long long)j * pos); }
};

// Pre-processing of one tile: builds the complex FFT input of every line in `buf`.  The kind is
// uniform, so each kind has its own loop; unrolling lets every thread keep several loads in flight.
template <class R, bool OY, int MC, class Src>
__device__ __noinline__ void pre_tile(const LineArgs& a, const Src src, int nl, cx<R>* buf) {
  const int M = MC ? MC : a.fp.M;
  const int N = a.N, ldm = a.ldm, kind = a.kind;
  const cx<R>* aux = reinterpret_cast<const cx<R>*>(a.aux);
  auto ldr = [&](auto b, int j) -> R { return src.ld(b, j); };
  auto ldc = [&](auto b, int j) -> cx<R> { return cx<R>{src.ld(b, j), src.ld(b + 1, j)}; };
  const FastDiv& fk = a.fd_kpre;
  if constexpr (!OY && MC > 0 && std::is_same<Src, SrcGlobal<R, typename Src::elem_t>>::value) {
    // x lines of a compile-time length: every thread reads runs of consecutive samples
    using SI = typename Src::elem_t;
    if (a.vec_ok) {
      if (kind == LK_DCT2 || kind == LK_DST2) {
        // u[4k..4k+3] -> z_k = (u_4k, u_4k+2), z_{M-1-k} = (u_4k+3, u_4k+1) (negated for DST-II)
        const bool dst = (kind == LK_DST2);
        using raw_t = typename Vec<R, SI>::raw_t;
        struct Raw { raw_t a, b; };
        for_items_xbt<R, MC, MC / 2, pre_batch(MC, 4)>(
            a, nl,
            [&](int L, int k) {
              const long long b = src.base(L) + 4LL * k;
              return Raw{Vec<R, SI>::raw(src.in, b), Vec<R, SI>::raw(src.in, b + 2)};
            },
            [&](int L, int k, const Raw& r) {
              R v[4];
              Vec<R, SI>::cvt(r.a, v);
              Vec<R, SI>::cvt(r.b, v + 2);
              buf[L * ldm + pad(k)] = cx<R>{v[0], v[2]};
              buf[L * ldm + pad((M - 1 - k))] = dst ? cx<R>{Ar<R>::neg(v[3]), Ar<R>::neg(v[1])} : cx<R>{v[3], v[1]};
            });
        return;
      }
      if (kind == LK_DCT4 || kind == LK_DST4) {
        // u[2n], u[2n+1] and u[N-2-2n], u[N-1-2n] -> z_n and z_{M-1-n}
        const bool c4 = (kind == LK_DCT4);
        for_items<false, MC / 2>(a, nl, fk, [&](int L, int n) {
          const long long b = src.base(L);
          R lo[2], hi[2];
          Vec<R, SI>::ld2(src.in, b + 2 * n, lo);
          Vec<R, SI>::ld2(src.in, b + (N - 2 - 2 * n), hi);
          cx<R> z0 = c4 ? cx<R>{lo[0], hi[1]} : cx<R>{hi[1], lo[0]};
          cx<R> z1 = c4 ? cx<R>{hi[0], lo[1]} : cx<R>{lo[1], hi[0]};
          buf[L * ldm + pad(n)] = cmul(z0, aux[n]);
          buf[L * ldm + pad((M - 1 - n))] = cmul(z1, aux[M - 1 - n]);
        });
        return;
      }
      if (kind == LK_R2C) {
        for_items<false, MC>(a, nl, fk, [&](int L, int k) {
          R v[2];
          Vec<R, SI>::ld2(src.in, src.base(L) + 2 * k, v);
          buf[L * ldm + pad(k)] = cx<R>{v[0], v[1]};
        });
        return;
      }
    }
    if (kind == LK_DCT3 || kind == LK_DST3) {
      // as the Hermitian-pair path below, with the four loads of up to two items issued together
      const cx<R>* w4 = aux + (M + 1);
      const bool c3 = (kind == LK_DCT3);
      struct Raw { SI y0, y1, y2, y3; };  // Y_k, Y_{N-k} (Y_N = 0), Y_{M-k}, Y_{M+k}
      for_items_xb<MC / 2 + 1, pre_batch(MC, 2)>(
          nl,
          [&](int L, int k) {
            const long long b = src.base(L);
            auto row = [&](int j) -> long long { return (long long)(c3 ? j : N - 1 - j) * src.pos; };
            Raw r;
            r.y0 = Io<R, SI>::raw(src.in, b + row(k));
            r.y1 = Io<R, SI>::raw(src.in, b + row(k > 0 ? N - k : 0));
            r.y2 = Io<R, SI>::raw(src.in, b + row(M - k));
            r.y3 = Io<R, SI>::raw(src.in, b + row(M + k));
            return r;
          },
          [&](int L, int k, const Raw& r) {
            const R y1 = k > 0 ? Io<R, SI>::cv(r.y1) : Ar<R>::zero();
            cx<R> Xk = cmulc(cx<R>{Io<R, SI>::cv(r.y0), Ar<R>::neg(y1)}, w4[k]);
            cx<R> Xm = cmulc(cx<R>{Io<R, SI>::cv(r.y2), Ar<R>::neg(Io<R, SI>::cv(r.y3))}, w4[M - k]);
            if (k == 0) { Xk.im = Ar<R>::zero(); Xm.im = Ar<R>::zero(); }
            cx<R> Xc = cconj(Xm);
            cx<R> E = cadd(Xk, Xc);
            cx<R> O = cmulc(csub(Xk, Xc), aux[k]);  // * conj(w_N^k)
            buf[L * ldm + pad(k)] = cx<R>{Ar<R>::sub(E.re, O.im), Ar<R>::add(E.im, O.re)};
            const int km = M - k;
            if (k > 0 && km != k) buf[L * ldm + pad(km)] = cx<R>{Ar<R>::add(E.re, O.im), Ar<R>::sub(O.re, E.im)};
          });
      return;
    }
  }
  if constexpr (OY) {
    // complex columns (C2C, FP32 kernels only: the double-float ones gained 5 % on C2C and lost 1 %
    // on the real kinds to the larger code): 16-byte loads of two adjacent complex lines per item
    if constexpr (std::is_same<R, float>::value) {
      if (a.vec_y == 2) {
        using SI = typename Src::elem_t;
        constexpr int VC = CVec<R, SI>::VC;
        const long long pos = src.pos;
        for_groups<VC, MC>(a, nl, fk, [&](int L0, int k, int nv) {
          cx<R> z[VC];
          CVec<R, SI>::ld(src.in, src.base(L0) + (long long)k * pos, nv, z);
#pragma unroll
          for (int v = 0; v < VC; v++)
            if (v < nv) buf[(L0 + v) * ldm + pad(k)] = z[v];
        });
        return;
      }
    }
    if (a.vec_y) {
      // real y lines of a contiguous tile row: V adjacent lines per item, 16-byte loads
      using SI = typename Src::elem_t;
      constexpr int V = VecN<R, SI>::V;
      const long long pos = src.pos;
      if (kind == LK_DCT2 || kind == LK_DST2) {
        const bool dst = (kind == LK_DST2);
        struct RawV { R v0[V], v1[V]; };
        auto ldv = [&](int L0, int k, int nv) -> RawV {
          const long long b = src.base(L0);
          const int j0 = 2 * k, j1 = 2 * k + 1;
          const int s0 = j0 < M ? 2 * j0 : 2 * N - 1 - 2 * j0;
          const int s1 = j1 < M ? 2 * j1 : 2 * N - 1 - 2 * j1;
          RawV r;
          ldn<R>(src.in, b + s0 * pos, nv, r.v0);
          ldn<R>(src.in, b + s1 * pos, nv, r.v1);
          return r;
        };
        auto stv = [&](int L0, int k, int nv, const RawV& r) {
          const int j0 = 2 * k, j1 = 2 * k + 1;
#pragma unroll
          for (int v = 0; v < V; v++) {
            if (v < nv) {
              R x0 = r.v0[v], x1 = r.v1[v];
              if (dst) {
                if (j0 >= M) x0 = Ar<R>::neg(x0);
                if (j1 >= M) x1 = Ar<R>::neg(x1);
              }
              buf[(L0 + v) * ldm + pad(k)] = cx<R>{x0, x1};
            }
          }
        };
        for_groups_yb<R, MC, V, MC>(a, nl, fk, ldv, stv);
        return;
      }
      if (kind == LK_DCT4 || kind == LK_DST4) {
        const bool c4 = (kind == LK_DCT4);
        for_groups<V, MC>(a, nl, fk, [&](int L0, int k, int nv) {
          const long long b = src.base(L0);
          R e[V], o[V];
          ldn<R>(src.in, b + (long long)(2 * k) * pos, nv, e);
          ldn<R>(src.in, b + (long long)(N - 1 - 2 * k) * pos, nv, o);
          const cx<R> w = aux[k];  // exp(-i pi (4k+1) / 4N)
#pragma unroll
          for (int v = 0; v < V; v++)
            if (v < nv) buf[(L0 + v) * ldm + pad(k)] = cmul(c4 ? cx<R>{e[v], o[v]} : cx<R>{o[v], e[v]}, w);
        });
        return;
      }
      if (kind == LK_DCT3 || kind == LK_DST3) {
        // as the scalar Hermitian-pair path below, V lines per item
        const cx<R>* w4 = aux + (M + 1);
        const bool c3 = (kind == LK_DCT3);
        for_groups_y<R, MC, V, (MC ? MC / 2 + 1 : 0)>(a, nl, fk, [&](int L0, int k, int nv) {
          const long long b = src.base(L0);
          auto row = [&](int j) -> long long { return (long long)(c3 ? j : N - 1 - j) * pos; };
          R y0[V], y1[V], y2[V], y3[V];  // Y_k, Y_{N-k} (Y_N = 0), Y_{M-k}, Y_{M+k}
          ldn<R>(src.in, b + row(k), nv, y0);
          if (k > 0) {
            ldn<R>(src.in, b + row(N - k), nv, y1);
          } else {
#pragma unroll
            for (int v = 0; v < V; v++) y1[v] = Ar<R>::zero();
          }
          ldn<R>(src.in, b + row(M - k), nv, y2);
          ldn<R>(src.in, b + row(M + k), nv, y3);
          const cx<R> wk = w4[k], wm = w4[M - k], ak = aux[k];
          const int km = M - k;
#pragma unroll
          for (int v = 0; v < V; v++) {
            if (v < nv) {
              cx<R> Xk = cmulc(cx<R>{y0[v], Ar<R>::neg(y1[v])}, wk);
              cx<R> Xm = cmulc(cx<R>{y2[v], Ar<R>::neg(y3[v])}, wm);
              if (k == 0) { Xk.im = Ar<R>::zero(); Xm.im = Ar<R>::zero(); }
              cx<R> Xc = cconj(Xm);
              cx<R> E = cadd(Xk, Xc);
              cx<R> O = cmulc(csub(Xk, Xc), ak);
              cx<R>* zl = buf + (L0 + v) * ldm;
              zl[pad(k)] = cx<R>{Ar<R>::sub(E.re, O.im), Ar<R>::add(E.im, O.re)};
              if (k > 0 && km != k) zl[pad(km)] = cx<R>{Ar<R>::add(E.re, O.im), Ar<R>::sub(O.re, E.im)};
            }
          }
        });
        return;
      }
    }
  }
  switch (kind) {
    case LK_R2C:
      for_items<OY, MC>(a, nl, fk, [&](int L, int k) {
        auto b = src.base(L);
        buf[L * ldm + pad(k)] = cx<R>{ldr(b, 2 * k), ldr(b, 2 * k + 1)};
      });
      break;
    case LK_DCT2:
    case LK_DST2: {
      // v_j = u_{2j} (j < M), u_{2N-1-2j} (j >= M); DST-II alternates the sign of odd samples
      const bool dst = (kind == LK_DST2);
      for_items<OY, MC>(a, nl, fk, [&](int L, int k) {
        auto b = src.base(L);
        int j0 = 2 * k, j1 = 2 * k + 1;
        int s0 = j0 < M ? 2 * j0 : 2 * N - 1 - 2 * j0;
        int s1 = j1 < M ? 2 * j1 : 2 * N - 1 - 2 * j1;
        R v0 = ldr(b, s0), v1 = ldr(b, s1);
        if (dst) {
          if (j0 >= M) v0 = Ar<R>::neg(v0);
          if (j1 >= M) v1 = Ar<R>::neg(v1);
        }
        buf[L * ldm + pad(k)] = cx<R>{v0, v1};
      });
      break;
    }
    case LK_DCT4:
    case LK_DST4: {
      const bool c4 = (kind == LK_DCT4);
      for_items<OY, MC>(a, nl, fk, [&](int L, int k) {
        auto b = src.base(L);
        R e = ldr(b, 2 * k), o = ldr(b, N - 1 - 2 * k);
        cx<R> z = c4 ? cx<R>{e, o} : cx<R>{o, e};
        buf[L * ldm + pad(k)] = cmul(z, aux[k]);  // exp(-i pi (4k+1) / 4N)
      });
      break;
    }
    case LK_C2C_F:
    case LK_C2C_I:
      for_items<OY, MC>(a, nl, fk, [&](int L, int k) { buf[L * ldm + pad(k)] = ldc(src.base(L), k); });
      break;
    case LK_C2R:
    case LK_DCT3:
    case LK_DST3: {
      // Hermitian pair (X_k, X_{M-k}) -> Z_k = E + i O, E = X_k + conj X_{M-k},
      // O = (X_k - conj X_{M-k}) exp(+2 pi i k / N); imaginary parts of X_0, X_M dropped.
      // The partner comes from the same two inputs: E_{M-k} = conj E and O_{M-k} = conj O, so
      // Z_{M-k} = (E.re + O.im) + i (O.re - E.im); item k <= M/2 writes Z_k and Z_{M-k}.
      // DCT-III/DST-III first form V_j = exp(+i pi j / 2N) (Y_j - i Y_{N-j}), Y_N = 0
      // (DST-III reads Y reversed).
      const cx<R>* w4 = aux + (M + 1);
      for_items<OY, (MC ? MC / 2 + 1 : 0)>(a, nl, fk, [&](int L, int k) {
        auto b = src.base(L);
        cx<R> Xk, Xm;
        if (kind == LK_C2R) {
          Xk = ldc(b, k);
          Xm = ldc(b, M - k);
        } else {
          auto Y = [&](int j) -> R {
            if (j >= N) return Ar<R>::zero();
            return ldr(b, kind == LK_DCT3 ? j : N - 1 - j);
          };
          cx<R> t0{Y(k), Ar<R>::neg(Y(N - k))};
          cx<R> t1{Y(M - k), Ar<R>::neg(Y(M + k))};
          Xk = cmulc(t0, w4[k]);
          Xm = cmulc(t1, w4[M - k]);
        }
        if (k == 0) { Xk.im = Ar<R>::zero(); Xm.im = Ar<R>::zero(); }
        cx<R> Xc = cconj(Xm);
        cx<R> E = cadd(Xk, Xc);
        cx<R> O = cmulc(csub(Xk, Xc), aux[k]);  // * conj(w_N^k)
        buf[L * ldm + pad(k)] = cx<R>{Ar<R>::sub(E.re, O.im), Ar<R>::add(E.im, O.re)};
        const int km = M - k;
        if (k > 0 && km != k) buf[L * ldm + pad(km)] = cx<R>{Ar<R>::add(E.re, O.im), Ar<R>::sub(O.re, E.im)};
      });
      break;
    }
    default: break;
  }
}

// Post-processing of one transformed tile: extracts the wanted transform from `buf` and writes
// it to global memory (line bases in s_bout).  One loop per (uniform) kind, as in pre_tile.
template <class R, class SO, bool OY, int MC>
__device__ __noinline__ void post_tile(const LineArgs& a, const cx<R>* buf, int nl, const long long* s_bout) {
  const int M = MC ? MC : a.fp.M;
  const int N = a.N, ldm = a.ldm, kind = a.kind;
  const cx<R>* aux = reinterpret_cast<const cx<R>*>(a.aux);
  SO* out = reinterpret_cast<SO*>(a.out);
  const long long op = a.out_pos;
  auto str = [&](long long b, int j, R v) { Io<R, SO>::st(out, b + (long long)j * op, v); };
  auto stc = [&](long long b, int j, cx<R> v) {
    long long o = b + (long long)j * op;
    Io<R, SO>::st(out, o, v.re);
    Io<R, SO>::st(out, o + 1, v.im);
  };
  const FastDiv& fk = a.fd_kpost;
  if constexpr (!OY && MC > 0) {
    if (a.vec_ok) {
      if (kind == LK_DCT3 || kind == LK_DST3) {
        // u[4k..4k+3] = (z_k.re, s z_{M-1-k}.im, z_k.im, s z_{M-1-k}.re), s = -1 for DST-III
        const bool dst = (kind == LK_DST3);
        for_items<false, MC / 2>(a, nl, fk, [&](int L, int k) {
          const long long b = s_bout[L] + 4LL * k;
          cx<R> z0 = buf[L * ldm + pad(k)], z1 = buf[L * ldm + pad((M - 1 - k))];
          if (dst) z1 = cx<R>{Ar<R>::neg(z1.re), Ar<R>::neg(z1.im)};
          R v[4] = {z0.re, z1.im, z0.im, z1.re};
          Vec<R, SO>::st2(out, b, v);
          Vec<R, SO>::st2(out, b + 2, v + 2);
        });
        return;
      }
      if (kind == LK_DCT4 || kind == LK_DST4) {
        // Y_2k = s_k.re, Y_{N-1-2k} = -+s_k.im; the partner k' = M-1-k fills Y_{2k+1}, Y_{N-2-2k}
        const bool c4 = (kind == LK_DCT4);
        for_items<false, MC / 2>(a, nl, fk, [&](int L, int k) {
          const long long b = s_bout[L];
          const int k1 = M - 1 - k;
          cx<R> s0 = cmul(buf[L * ldm + pad(k)], aux[M + k]);
          cx<R> s1 = cmul(buf[L * ldm + pad(k1)], aux[M + k1]);
          R i0 = c4 ? Ar<R>::neg(s0.im) : s0.im, i1 = c4 ? Ar<R>::neg(s1.im) : s1.im;
          R lo[2] = {s0.re, i1}, hi[2] = {s1.re, i0};
          Vec<R, SO>::st2(out, b + 2 * k, lo);
          Vec<R, SO>::st2(out, b + (N - 2 - 2 * k), hi);
        });
        return;
      }
      if (kind == LK_C2R) {
        for_items<false, MC>(a, nl, fk, [&](int L, int k) {
          cx<R> z = buf[L * ldm + pad(k)];
          R v[2] = {z.re, z.im};
          Vec<R, SO>::st2(out, s_bout[L] + 2 * k, v);
        });
        return;
      }
    }
  }
  if constexpr (OY) {
    // complex columns (C2C, FP32 kernels only, as in pre_tile): 16-byte stores of two adjacent
    // complex lines per item
    if constexpr (std::is_same<R, float>::value) {
      if (a.vec_y == 2) {
        constexpr int VC = CVec<R, SO>::VC;
        for_groups<VC, MC>(a, nl, fk, [&](int L0, int k, int nv) {
          cx<R> z[VC];
#pragma unroll
          for (int v = 0; v < VC; v++) z[v] = (v < nv) ? buf[(L0 + v) * ldm + pad(k)] : cx<R>{Ar<R>::zero(), Ar<R>::zero()};
          CVec<R, SO>::st(out, s_bout[L0] + (long long)k * op, nv, z);
        });
        return;
      }
    }
    if (a.vec_y) {
      // real y lines of a contiguous tile row: V adjacent lines per item, 16-byte stores
      constexpr int V = VecN<R, SO>::V;
      if (kind == LK_DCT2 || kind == LK_DST2) {
        // as the scalar Hermitian-pair path below, V lines per item
        const bool dst = (kind == LK_DST2);
        for_groups_y<R, MC, V, (MC ? MC / 2 + 1 : 0)>(a, nl, fk, [&](int L0, int k, int nv) {
          const long long b = s_bout[L0];
          const int km = M - k;
          const cx<R> ak = aux[k], wk = aux[M + 1 + k], wm = aux[M + 1 + km];
          R r0[V], r1[V], r2[V], r3[V];
#pragma unroll
          for (int v = 0; v < V; v++) {
            if (v < nv) {
              const cx<R>* zl = buf + (L0 + v) * ldm;
              cx<R> Zk = zl[pad(k)];
              cx<R> Zc = cconj(zl[pad(k == 0 ? 0 : km)]);
              cx<R> E = chalf(cadd(Zk, Zc));
              cx<R> dd = csub(Zk, Zc);
              cx<R> P = cmul(chalf(cx<R>{dd.im, Ar<R>::neg(dd.re)}), ak);
              cx<R> W0 = cmul(cadd(E, P), wk);
              cx<R> W1 = cmul(cconj(csub(E, P)), wm);
              r0[v] = W0.re; r1[v] = Ar<R>::neg(W0.im);
              r2[v] = W1.re; r3[v] = Ar<R>::neg(W1.im);
            } else {
              r0[v] = r1[v] = r2[v] = r3[v] = Ar<R>::zero();
            }
          }
          auto i0 = [&](int kk) -> long long { return (long long)(dst ? N - 1 - kk : kk) * op; };
          auto i1 = [&](int kk) -> long long { return (long long)(dst ? kk - 1 : N - kk) * op; };
          stn<R>(out, b + i0(k), nv, r0);
          if (k >= 1 && k < M) stn<R>(out, b + i1(k), nv, r1);
          if (km != k) {
            stn<R>(out, b + i0(km), nv, r2);
            if (km >= 1 && km < M) stn<R>(out, b + i1(km), nv, r3);
          }
        });
        return;
      }
      if (kind == LK_DCT3 || kind == LK_DST3) {
        const bool dst = (kind == LK_DST3);
        for_groups_y<R, MC, V, MC>(a, nl, fk, [&](int L0, int k, int nv) {
          const long long b = s_bout[L0];
          const int j0 = 2 * k, j1 = 2 * k + 1;
          const int s0 = j0 < M ? 2 * j0 : 2 * N - 1 - 2 * j0;
          const int s1 = j1 < M ? 2 * j1 : 2 * N - 1 - 2 * j1;
          R r0[V], r1[V];
#pragma unroll
          for (int v = 0; v < V; v++) {
            cx<R> z = (v < nv) ? buf[(L0 + v) * ldm + pad(k)] : cx<R>{Ar<R>::zero(), Ar<R>::zero()};
            r0[v] = (dst && j0 >= M) ? Ar<R>::neg(z.re) : z.re;
            r1[v] = (dst && j1 >= M) ? Ar<R>::neg(z.im) : z.im;
          }
          stn<R>(out, b + (long long)s0 * op, nv, r0);
          stn<R>(out, b + (long long)s1 * op, nv, r1);
        });
        return;
      }
      if (kind == LK_DCT4 || kind == LK_DST4) {
        const bool c4 = (kind == LK_DCT4);
        for_groups<V, MC>(a, nl, fk, [&](int L0, int k, int nv) {
          const long long b = s_bout[L0];
          const cx<R> w = aux[M + k];  // exp(-i pi k / N)
          R r0[V], r1[V];
#pragma unroll
          for (int v = 0; v < V; v++) {
            cx<R> sv = (v < nv) ? cmul(buf[(L0 + v) * ldm + pad(k)], w) : cx<R>{Ar<R>::zero(), Ar<R>::zero()};
            r0[v] = sv.re;
            r1[v] = c4 ? Ar<R>::neg(sv.im) : sv.im;
          }
          stn<R>(out, b + (long long)(2 * k) * op, nv, r0);
          stn<R>(out, b + (long long)(N - 1 - 2 * k) * op, nv, r1);
        });
        return;
      }
    }
  }
  switch (kind) {
    case LK_R2C:
    case LK_DCT2:
    case LK_DST2: {
      // X_k = E_k + w_N^k O_k from the Hermitian pair (Z_k, Z_{M-k}), E_k = (Z_k + conj Z_{M-k})/2,
      // O_k = (Z_k - conj Z_{M-k})/2i.  The partner needs no second pass: E_{M-k} = conj E_k,
      // O_{M-k} = conj O_k and w_N^{M-k} = -conj w_N^k give X_{M-k} = conj(E_k - w_N^k O_k); item
      // k <= M/2 emits X_k and X_{M-k} (k = 0: X_0 and X_M).  DCT-II: W = exp(-i pi k/2N) X_k,
      // Y_k = Re W, Y_{N-k} = -Im W; DST-II writes the DCT-II of the sign-alternated line reversed.
      for_items_x<R, OY, MC, (MC ? MC / 2 + 1 : 0)>(a, nl, fk, [&](int L, int k) {
        const long long b = s_bout[L];
        const cx<R>* zl = buf + L * ldm;
        const int km = M - k;
        cx<R> Zk = zl[pad(k)];
        cx<R> Zm = zl[pad(k == 0 ? 0 : km)];
        cx<R> Zc = cconj(Zm);
        cx<R> E = chalf(cadd(Zk, Zc));
        cx<R> dd = csub(Zk, Zc);
        cx<R> O = chalf(cx<R>{dd.im, Ar<R>::neg(dd.re)});  // (Zk - conj Zm) / (2i)
        cx<R> P = cmul(O, aux[k]);                         // w_N^k O
        auto emit = [&](int kk, cx<R> X) {
          if (kind == LK_R2C) { stc(b, kk, X); return; }
          cx<R> W = cmul(X, aux[M + 1 + kk]);              // exp(-i pi kk / 2N)
          int i0 = kk, i1 = N - kk;
          if (kind == LK_DST2) { i0 = N - 1 - kk; i1 = kk - 1; }
          str(b, i0, W.re);
          if (kk >= 1 && kk < M) str(b, i1, Ar<R>::neg(W.im));
        };
        emit(k, cadd(E, P));
        if (km != k) emit(km, cconj(csub(E, P)));
      });
      break;
    }
    case LK_DCT4:
    case LK_DST4: {
      const bool c4 = (kind == LK_DCT4);
      for_items<OY, MC>(a, nl, fk, [&](int L, int k) {
        const long long b = s_bout[L];
        cx<R> s = cmul(buf[L * ldm + pad(k)], aux[M + k]);  // exp(-i pi k / N)
        str(b, 2 * k, s.re);
        str(b, N - 1 - 2 * k, c4 ? Ar<R>::neg(s.im) : s.im);
      });
      break;
    }
    case LK_C2C_F:
    case LK_C2C_I:
      for_items<OY, MC>(a, nl, fk, [&](int L, int k) { stc(s_bout[L], k, buf[L * ldm + pad(k)]); });
      break;
    case LK_C2R:
      for_items<OY, MC>(a, nl, fk, [&](int L, int k) {
        const long long b = s_bout[L];
        cx<R> z = buf[L * ldm + pad(k)];
        str(b, 2 * k, z.re);
        str(b, 2 * k + 1, z.im);
      });
      break;
    case LK_DCT3:
    case LK_DST3: {
      // u_{sigma(j)} = v_j with sigma the Makhoul order (DST-III: signs alternate)
      const bool dst = (kind == LK_DST3);
      for_items<OY, MC>(a, nl, fk, [&](int L, int k) {
        const long long b = s_bout[L];
        cx<R> z = buf[L * ldm + pad(k)];
        int j0 = 2 * k, j1 = 2 * k + 1;
        int s0 = j0 < M ? 2 * j0 : 2 * N - 1 - 2 * j0;
        int s1 = j1 < M ? 2 * j1 : 2 * N - 1 - 2 * j1;
        R v0 = z.re, v1 = z.im;
        if (dst) {
          if (j0 >= M) v0 = Ar<R>::neg(v0);
          if (j1 >= M) v1 = Ar<R>::neg(v1);
        }
        str(b, s0, v0);
        str(b, s1, v1);
      });
      break;
    }
    default: break;
  }
}

// Register caps (measured): FP32 48 (ten 128-thread CTAs per SM); double-float 64 (eight), except
// the warp-per-line y kernels of 512-point lines, which hold 16 values per thread (80: the
// double-float one spills 144 bytes per thread and is still faster than at 96 or 72).  None of the other
// compile-time-length kernels spills.  The run-time-length kernels get 64 (FP32) and 128
// (double-float).
template <class R, int MC, bool OY> struct MaxRegs {
  static constexpr bool RT = MC <= 0;  // run-time lengths
  static constexpr int v = std::is_same<R, float>::value ? (RT ? 64 : 48)
                                                         : (RT ? 128 : ((OY && MC == 512) ? 80 : 64));
};

// One tile per CTA (x: lpc consecutive rows; y: one plane x tx columns).
template <class R, class SI, class SO, bool OY, int MC>
__global__ void __maxnreg__((MaxRegs<R, MC, OY>::v)) k_lines(const LineArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const LineArgs& a = args;
  // MC > 0: compile-time length; 0: run-time length (radices 2, 3, 4, 8); -1: run-time length
  // with radix-5/7 stages as well
  constexpr int MCT = MC > 0 ? MC : 0;
  const int M = MCT ? MCT : a.fp.M;
  const int ldm = a.ldm;
  cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tws = buf + (size_t)a.lpc * ldm;
  // per-line base offsets of the tile (input, output), after the twiddles
  long long* s_bin = reinterpret_cast<long long*>(tws + M);
  long long* s_bout = s_bin + a.lpc;
  const cx<R>* twg = reinterpret_cast<const cx<R>*>(a.tw);
  // stage twiddles: w_M^j, j < M (run-time lengths) or the per-stage table of fft_lines_ct.
  // Asynchronous copies (cp.async), waited for after the pre-processing: their latency then
  // overlaps the line loads instead of preceding them.
  for (int i = threadIdx.x; i < M; i += blockDim.x) cp_async_cx(tws + i, twg + i);
  cp_async_commit();
  const int kind = a.kind;
  const bool inv = (kind == LK_C2R || kind == LK_C2C_I || kind == LK_DCT3 || kind == LK_DST3);
  int line0, nl;
  if (!OY) {
    line0 = (int)blockIdx.x * a.lpc;
    nl = min(a.lpc, a.nlines - line0);
  } else {
    const int plane = (int)a.fd_nblk.div(blockIdx.x);
    const int blk = (int)blockIdx.x - plane * a.nblk;
    const int c0 = blk * a.tx;
    line0 = plane * a.lines_per_plane + c0 * a.parts;
    nl = min(a.tx, a.ncols - c0) * a.parts;
  }
  for (int L = threadIdx.x; L < nl; L += blockDim.x) {
    s_bin[L] = line_base(a, (unsigned)(line0 + L), false);
    s_bout[L] = line_base(a, (unsigned)(line0 + L), true);
  }
  __syncthreads();
  pre_tile<R, OY, MCT>(a, SrcGlobal<R, SI>{reinterpret_cast<const SI*>(a.in), s_bin, (long long)a.in_pos}, nl, buf);
  cp_async_wait_all();
  __syncthreads();
  if constexpr (MC > 0) {
    // double-float lines of 256+ complex points: radix-8 stages share one copy of the butterfly
    // (measured faster there; the shorter lengths keep fully compile-time stages)
    constexpr int VPT = ct_values_per_thread(MC, OY, std::is_same<R, df>::value);
    if constexpr (std::is_same<R, df>::value && MC >= 256 && ct_pow2(MC)) {
      if (inv) fft_lines_lp<R, true, MC, VPT>(buf, nl, ldm, tws);
      else fft_lines_lp<R, false, MC, VPT>(buf, nl, ldm, tws);
    } else {
      if (inv) fft_lines_ct<R, true, MC, VPT>(buf, nl, ldm, tws);
      else fft_lines_ct<R, false, MC, VPT>(buf, nl, ldm, tws);
    }
    __syncthreads();  // warp teams synchronised only themselves; post-processing reads every line
  } else {
    if (inv) fft_lines<R, true, (MC < 0)>(buf, nl, ldm, a.fp, tws);
    else fft_lines<R, false, (MC < 0)>(buf, nl, ldm, a.fp, tws);
    if (a.fp.nst == 0) __syncthreads();
  }
  post_tile<R, SO, OY, MCT>(a, buf, nl, s_bout);
}

template <class R, class SI, class SO, bool OY, int MC>
cudaError_t launch_lines_k(const LineArgs& a, int threads, cudaStream_t st) {
  auto k = k_lines<R, SI, SO, OY, MC>;
  // dynamic shared memory above 48 KB must be opted into, per device; plans keep it <= 200 KB.
  // One bit per device ordinal (below 64; higher ordinals set the attribute on every launch).
  static std::atomic<unsigned long long> attr_done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (!bit || !(attr_done.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_done.fetch_or(bit, std::memory_order_release);
  }
  const size_t sm = ((size_t)a.lpc * a.ldm + (size_t)a.fp.M) * sizeof(cx<R>) + 2 * (size_t)a.lpc * sizeof(long long);
  k<<<a.ntiles, threads, sm, st>>>(a);
  return cudaGetLastError();
}

// storage codes of the launchers
enum { ST_F64 = 0, ST_F32 = 1, ST_SPILL = 2 };

// Pick the instantiation for (orientation, input/output storage) and the FFT length.
template <class R, class SP, int MC>
cudaError_t dispatch_io(const LineArgs& a, int oy, int sin, int sout, int threads, cudaStream_t st) {
  if (oy) {
    if (sin == ST_SPILL && sout == ST_SPILL) return launch_lines_k<R, SP, SP, true, MC>(a, threads, st);
    return cudaErrorInvalidValue;
  }
  if (sin == ST_F64 && sout == ST_SPILL) return launch_lines_k<R, double, SP, false, MC>(a, threads, st);
  if (sin == ST_SPILL && sout == ST_F64) return launch_lines_k<R, SP, double, false, MC>(a, threads, st);
  if (sin == ST_SPILL && sout == ST_SPILL) return launch_lines_k<R, SP, SP, false, MC>(a, threads, st);
  if (std::is_same<R, float>::value) {
    // FP32 I/O: the spill type is float as well
    if ((sin == ST_F32 && sout == ST_SPILL) || (sin == ST_SPILL && sout == ST_F32))
      return launch_lines_k<R, SP, SP, false, MC>(a, threads, st);
  }
  return cudaErrorInvalidValue;
}

// Instantiation groups (one translation unit each, compiled in parallel): compile-time lengths
// {8, 16, 32}, {64, 128, 256}, {512, 1024}, {24, 48, 96} and {192, 384, 768}, plus the
// run-time-length kernels (without and with radix-5/7 stages).  Each returns cudaErrorNotSupported when the length is not in its group.
#define PP_LINES_GROUP_DECL(name) \
  cudaError_t name(const LineArgs& a, int oy, int sin, int sout, int threads, cudaStream_t st)
PP_LINES_GROUP_DECL(lines_df_tiny);
PP_LINES_GROUP_DECL(lines_df_small);
PP_LINES_GROUP_DECL(lines_df_large);
PP_LINES_GROUP_DECL(lines_df_ct3a);
PP_LINES_GROUP_DECL(lines_df_ct3b);
PP_LINES_GROUP_DECL(lines_df_any);
PP_LINES_GROUP_DECL(lines_df_any57);
PP_LINES_GROUP_DECL(lines_f32_tiny);
PP_LINES_GROUP_DECL(lines_f32_small);
PP_LINES_GROUP_DECL(lines_f32_large);
PP_LINES_GROUP_DECL(lines_f32_ct3a);
PP_LINES_GROUP_DECL(lines_f32_ct3b);
PP_LINES_GROUP_DECL(lines_f32_any);
PP_LINES_GROUP_DECL(lines_f32_any57);

}  // namespace pp
