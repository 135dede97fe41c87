// pp_zpart.cu -- the z tridiagonal solve of non-periodic z with every line split into chunks
// (Sec. "Solution of the Resulting Tridiagonal Matrices"; the parallel alternatives to the
// sequential Thomas sweep of Sec. "Cyclic Reduction Technique" / "Parallel Cyclic Reduction").
//
// The Thomas solve of a mode (pp_zsolve.cu) is two first-order linear recurrences over the rows,
// with the plan's precomputed multipliers w_k:
//     forward   g_k = (s d_k - g_{k-1}) w_k = a_k g_{k-1} + w_k s d_k,      a_k = -w_k, g_{-1} = 0,
//     backward  u_k = g_k - w_k u_{k+1}     = a_k u_{k+1} + g_k,            u_n = 0.
// One thread per line runs them in sequence: with few modes and long lines (the setting of the
// paper's solver comparison, 64 x 64 modes and up to 4095 rows) the GPU has too few threads for
// that.  Here a line is split into P chunks of M consecutive rows, one thread per chunk, and each
// recurrence is solved in three steps:
//   1. every thread runs the recurrence over its chunk from a zero carry, keeping the local
//      values and the chunk's affine map x_out = A x_in + B (A the product of its a_k);
//   2. the maps of the P chunks of a line are composed by recursive doubling (Kogge-Stone: at
//      level j every chunk composes its map with the one 2^j chunks before it), with warp
//      shuffles inside a warp's run of chunks and one shared-memory exchange of the warps' totals,
//      which gives each chunk its true carry;
//   3. every thread adds (product of a_i up to row k) x carry to its local values.
// The multipliers and the order of the per-row operations are those of the Thomas sweeps, so the
// result is the Thomas result up to the rounding of the chunk products; unlike cyclic reduction
// applied to the rows of the tridiagonal system, nothing forms the reduced systems' diagonals,
// whose distance from weak diagonal dominance (about the square of the lowest wavenumber)
// double-float coefficients would not keep.
//
// The M values of a thread stay in registers between the steps.  A CTA takes G adjacent real slots (consecutive threads: consecutive slots, so
// every row access of a warp is a few contiguous segments) x P chunks; G P <= 512.  Padding slots
// take part in the scans with their maps unused; the singular mode's column is left untouched
// (the plan solves it with the pinned Thomas sweep afterwards).
//
// Arithmetic: double-float (pp_arith.cuh) on the plan's spill type.  Range report: pp_range.cuh.
#include "pp_range.cuh"
#include "pp_zmul.cuh"

namespace pp {

__device__ __forceinline__ df zp_ld(const float2* p) { const float2 v = *p; return df{v.x, v.y}; }
__device__ __forceinline__ df zp_ld(const float* p) { return df{*p, 0.0f}; }
__device__ __forceinline__ void zp_st(float2* p, df v) { *p = make_float2(v.hi, v.lo); }
__device__ __forceinline__ void zp_st(float* p, df v) { *p = df_to_f32(v); }
__device__ __forceinline__ df zp_f2(float2 v) { return df{v.x, v.y}; }
__device__ __forceinline__ df zp_f2(const float* v) { return df{v[0], v[1]}; }

// (A, B) pairs of one carry's segment totals: up to 16 warps x 8 lines, two words each
constexpr int kZpAgg = 2 * 16 * 8;

// Composition of chunk maps x -> A x + B: (X o Y)(x) = X(Y(x)) = (A_X A_Y) x + (A_X B_Y + B_X).
__device__ __forceinline__ void zp_compose(df& A, df& B, df Ay, df By) {
  B = A * By + B;
  A = A * Ay;
}
__device__ __forceinline__ df zp_shfl(df v, int delta, bool up) {
  return up ? df{__shfl_up_sync(0xffffffffu, v.hi, delta), __shfl_up_sync(0xffffffffu, v.lo, delta)}
            : df{__shfl_down_sync(0xffffffffu, v.hi, delta), __shfl_down_sync(0xffffffffu, v.lo, delta)};
}

// Carry of every chunk from the chunk maps of its line, by recursive doubling in two levels.  A warp
// holds CW = 32 / G consecutive chunks of each of the CTA's G lines (lane = chunk-in-warp x G +
// line), one segment per line; the warp's segments are scanned with shuffles (log2 CW levels: at
// level o a chunk composes its map with the one o chunks nearer the start of the recurrence), the
// segment totals are exchanged through shared memory (one barrier), and each chunk composes the
// totals of the segments before its own.
// dir = +1 (forward recurrence, starting at chunk 0): returns the value entering the chunk, the
// output of chunk c - 1 (0 for chunk 0).  dir = -1 (backward recurrence, starting at the last
// chunk): the output of chunk c + 1 (0 for the last).
// agg: NS x G pairs of (A, B), NS = warps of the CTA.  Every thread calls it; chunks past the line
// (c >= P) hold the identity map, which composes away.
__device__ __forceinline__ df zp_carry(df A, df B, float2* agg, int c, int col, int G, int lgG, int dir) {
  const int lane = (int)threadIdx.x & 31;
  const int cw = 32 >> lgG;          // chunks per warp and line
  const int ci = lane >> lgG;        // chunk within the warp's segment
  const int seg = (int)threadIdx.x >> 5;
  const int nseg = ((int)blockDim.x + 31) >> 5;
  const bool fwd = dir > 0;
  // 1. inclusive scan within the segment
  for (int o = 1; o < cw; o <<= 1) {
    const df An = zp_shfl(A, o * G, fwd), Bn = zp_shfl(B, o * G, fwd);
    if (fwd ? (ci >= o) : (ci + o < cw)) zp_compose(A, B, An, Bn);
  }
  // the inclusive map of the neighbouring chunk nearer the start (same segment unless at its edge)
  const df An1 = zp_shfl(A, G, fwd), Bn1 = zp_shfl(B, G, fwd);
  // 2. segment totals: the last chunk of a forward segment, the first of a backward one
  float2* sA = agg;
  float2* sB = agg + nseg * G;
  if (fwd ? (ci == cw - 1) : (ci == 0)) {
    sA[seg * G + col] = make_float2(A.hi, A.lo);
    sB[seg * G + col] = make_float2(B.hi, B.lo);
  }
  __syncthreads();
  // 3. L: the composition of the segments before this one (forward: segments 0 .. seg-1, applied
  // in that order; backward: the last segment down to seg+1)
  df La = df{1.f, 0.f}, Lb = df{0.f, 0.f};
  for (int t = 0; t < (fwd ? seg : nseg - 1 - seg); t++) {
    const int j = fwd ? t : nseg - 1 - t;
    df Aj = zp_f2(sA[j * G + col]), Bj = zp_f2(sB[j * G + col]);
    zp_compose(Aj, Bj, La, Lb);  // L = Agg_j o L
    La = Aj;
    Lb = Bj;
  }
  // the carry: the neighbour's output, its segment map applied to L's output (at the segment's
  // edge, L's output itself)
  const bool edge = fwd ? (ci == 0) : (ci == cw - 1);
  return edge ? Lb : An1 * Lb + Bn1;
}

// The multiplier of row k (table prefix, converged value, last row), as stored (pp_zmul.cuh).
struct ZpW {
  const float2* wt;
  int wlen, n;
  bool plus1;  // the table holds w but the thread runs the near -1 form: convert to 1 + w
  df winf, wlast;
  __device__ __forceinline__ df operator()(int k) const {
    if (k == n - 1) return wlast;
    if (k < wlen) {
      const df x = zp_f2(__ldg(wt + k));
      return plus1 ? x + df{1.f, 0.f} : x;
    }
    return winf;
  }
};

// chunks of 16 rows keep their multipliers in registers across the four passes (measured: at 8 rows
// the extra registers halve the resident CTAs, at 32 they spill)
template <int M> struct ZpCacheW { static constexpr bool v = M == 16; };

// The four passes over a thread's M rows, with the chunk's multipliers wv loaded once (FAST: every
// row past the table prefix and not the last row, so w = winf throughout and wv is not read).  No
// barrier inside: a CTA's threads may take different variants.
// 1. forward recurrence from a zero carry: v = local g, (A, B) = the chunk's map
template <int M, bool N1, bool FAST>
__device__ __forceinline__ void zp_fwd(df (&v)[M], df& A, df& B, const ZpW& W, const df (&wv)[M], int k0, df scale, float& dmax) {
#pragma unroll
  for (int i = 0; i < M; i++) {
    const int k = k0 + i;
    if (FAST || k < W.n) {
      const df d = v[i] * scale;
      track(dmax, d.hi);
      const df w = FAST ? W.winf : (ZpCacheW<M>::v ? wv[i] : W(k));
      B = zw_mul<N1>(d - B, w);
      A = zw_neg_mul<N1>(A, w);
      v[i] = B;
    }
  }
}
// 2. g_k = local g_k + (a_k0 ... a_k) g_in
template <int M, bool N1, bool FAST>
__device__ __forceinline__ void zp_fwd_fix(df (&v)[M], df gin, const ZpW& W, const df (&wv)[M], int k0) {
  df Pk = df{1.f, 0.f};
#pragma unroll
  for (int i = 0; i < M; i++) {
    const int k = k0 + i;
    if (FAST || k < W.n) {
      Pk = zw_neg_mul<N1>(Pk, FAST ? W.winf : (ZpCacheW<M>::v ? wv[i] : W(k)));
      v[i] = v[i] + Pk * gin;
    }
  }
}
// 3. back substitution u_k = g_k - w_k u_{k+1} from a zero carry above the chunk
template <int M, bool N1, bool FAST>
__device__ __forceinline__ void zp_bwd(df (&v)[M], df& A, df& B, const ZpW& W, const df (&wv)[M], int k0) {
#pragma unroll
  for (int i = M - 1; i >= 0; i--) {
    const int k = k0 + i;
    if (FAST || k < W.n) {
      const df w = FAST ? W.winf : (ZpCacheW<M>::v ? wv[i] : W(k));
      B = zw_sub<N1>(v[i], w, B);
      A = zw_neg_mul<N1>(A, w);
      v[i] = B;
    }
  }
}
// 4. u_k = local u_k + (a_k ... a_end) u_in
template <int M, bool N1, bool FAST>
__device__ __forceinline__ void zp_bwd_fix(df (&v)[M], df uin, const ZpW& W, const df (&wv)[M], int k0) {
  df Qk = df{1.f, 0.f};
#pragma unroll
  for (int i = M - 1; i >= 0; i--) {
    const int k = k0 + i;
    if (FAST || k < W.n) {
      Qk = zw_neg_mul<N1>(Qk, FAST ? W.winf : (ZpCacheW<M>::v ? wv[i] : W(k)));
      v[i] = v[i] + Qk * uin;
    }
  }
}

#define ZP_DISPATCH(fn, ...)                                       \
  do {                                                             \
    if (fast) {                                                    \
      if (n1) fn<M, true, true>(__VA_ARGS__);                      \
      else fn<M, false, true>(__VA_ARGS__);                        \
    } else {                                                       \
      if (n1) fn<M, true, false>(__VA_ARGS__);                     \
      else fn<M, false, false>(__VA_ARGS__);                       \
    }                                                              \
  } while (0)

template <class S, int M>
__global__ void __launch_bounds__(512) k_zpart(const ZArgs a, int G, int lgG, int P) {
  __shared__ float2 zp_sm[2 * kZpAgg];  // segment totals of the forward and the backward carries
  const int tid = (int)threadIdx.x;
  const int col = tid & (G - 1);
  const int c = tid >> lgG;
  const long long s = (long long)blockIdx.x * G + col;
  const int n = a.nz;
  const long long PL = a.plane;

  // the slot's mode; padding slots, the singular mode and the threads that round the CTA up to
  // whole warps (c >= P) do no work but join every barrier
  const bool inb = c < P;
  bool live = inb && s < a.nreal;
  const ZMode* m = nullptr;
  if (live) {
    const unsigned row = a.fd_row.div((unsigned)s);
    const int cr = (int)(s - (long long)row * a.row_reals);
    live = cr < a.row_valid;
    if (live) {
      m = a.modes + ((long long)row * a.row_modes + (a.cplx ? (cr >> 1) : cr));
      live = !(m->flags & ZF_SINGULAR);
    }
  }
  ZpW W;
  W.wt = a.wtab;
  W.wlen = 0;
  W.n = n;
  W.winf = df{0.f, 0.f};
  W.wlast = df{0.f, 0.f};
  bool mine = false;
  if (live) {
    W.winf = zp_f2(m->winf);
    W.wlast = zp_f2(m->wlast);
    W.wlen = m->wlen;
    W.wt = a.wtab + m->woff;
    mine = (m->flags & ZF_NEAR1) != 0;
  }
  // a warp runs the near -1 form when any of its modes needs it (the others convert their w)
  const bool n1 = __any_sync(0xffffffffu, mine);
  W.plus1 = n1 && !mine;
  if (W.plus1) {
    W.winf = W.winf + df{1.f, 0.f};
    W.wlast = W.wlast + df{1.f, 0.f};
  }
  const int k0 = c * M;
  // a chunk past the multiplier prefix that does not hold the last row uses winf throughout
  const bool fast = k0 >= W.wlen && k0 + M < n;
  const df scale = df{a.scale[0], a.scale[1]};
  S* base = reinterpret_cast<S*>(a.data) + s;
  float dmax = 0.0f, umax = 0.0f;
  // the chunk's multipliers, loaded once for the four passes (chunks in the table prefix)
  df wv[M];
#pragma unroll
  for (int i = 0; i < M; i++) wv[i] = (ZpCacheW<M>::v && !fast && k0 + i < n) ? W(k0 + i) : W.winf;

  df v[M];
#pragma unroll
  for (int i = 0; i < M; i++) {
    const int k = k0 + i;
    v[i] = (live && k < n) ? zp_ld(base + (long long)k * PL) : df{0.f, 0.f};
  }

  // forward recurrence: local pass, carries by recursive doubling, fix-up
  df A = df{1.f, 0.f}, B = df{0.f, 0.f};
  ZP_DISPATCH(zp_fwd, v, A, B, W, wv, k0, scale, dmax);
  const df gin = zp_carry(A, B, zp_sm, c, col, G, lgG, +1);
  if (inb && c > 0) ZP_DISPATCH(zp_fwd_fix, v, gin, W, wv, k0);

  // back substitution: the same three steps from the top of each chunk
  A = df{1.f, 0.f};
  B = df{0.f, 0.f};
  ZP_DISPATCH(zp_bwd, v, A, B, W, wv, k0);
  const df uin = zp_carry(A, B, zp_sm + kZpAgg, c, col, G, lgG, -1);
  if (c + 1 < P) ZP_DISPATCH(zp_bwd_fix, v, uin, W, wv, k0);
  if (live) {
#pragma unroll
    for (int i = 0; i < M; i++) {
      const int k = k0 + i;
      if (k < n) {
        track(umax, v[i].hi);
        zp_st(base + (long long)k * PL, v[i]);
      }
    }
  }
  range_report(a.rstat, a.dmin, a.umax, gridDim.x, dmax, umax);
}
#undef ZP_DISPATCH

// Chunk count P = ceil(nz / M) and slots per CTA G (a power of two, G P <= 512, G <= 8; the CTA
// is G P threads rounded up to whole warps); returns false when a line needs more than 512 chunks.
bool zpart_shape(int nz, int M, int* G, int* lgG, int* P) {
  const int p = (nz + M - 1) / M;
  if (p > 512) return false;
  int g = 8, lg = 3;
  while (g > 1 && g * p > 512) { g >>= 1; lg--; }
  *G = g; *lgG = lg; *P = p;
  return true;
}

template <class S, int M>
static cudaError_t launch_zpart_t(const ZArgs& a, cudaStream_t st) {
  int G, lgG, P;
  if (!zpart_shape(a.nz, M, &G, &lgG, &P)) return cudaErrorInvalidConfiguration;
  const long long grid = (a.nreal + G - 1) / G;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const int threads = (G * P + 31) / 32 * 32;  // whole warps (the scans and the range report shuffle)
  k_zpart<S, M><<<(unsigned)grid, threads, 0, st>>>(a, G, lgG, P);
  return cudaGetLastError();
}

cudaError_t launch_zpart_impl(const ZArgs& a, bool df_spill, int M, cudaStream_t st) {
  switch (M) {
    case 8: return df_spill ? launch_zpart_t<float2, 8>(a, st) : launch_zpart_t<float, 8>(a, st);
    case 16: return df_spill ? launch_zpart_t<float2, 16>(a, st) : launch_zpart_t<float, 16>(a, st);
    case 32: return df_spill ? launch_zpart_t<float2, 32>(a, st) : launch_zpart_t<float, 32>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pp
