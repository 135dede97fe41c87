// pp_lines.cu -- batched line transforms along x (contiguous lines) and y (strided columns).
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
// Execution: persistent CTAs walk over tiles of `lpc` lines.  The raw input of the next tile
// is copied global -> shared memory with cp.async (16-byte chunks when the layout allows)
// while the current tile is transformed, so global-load latency overlaps the FFT.  An x tile
// is one contiguous run of rows; a y tile is a block of `tx` adjacent columns of one plane,
// staged row by row (each row segment is a contiguous, coalesced run).  Pre-processing reads
// the staged tile, the FFT runs in place in shared memory, post-processing writes straight to
// global memory (x: consecutive threads along a line; y: consecutive threads across columns).
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "pp_internal.h"

namespace pp {

// ------------------------------------------------------------------ cp.async helpers
template <int CH> __device__ __forceinline__ void cp_async(void* smem_dst, const void* gsrc) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  if (CH == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gsrc), "n"(CH) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// plain loads from the staged tile (shared memory) into the arithmetic type
template <class R, class S> struct SmemLd;
template <> struct SmemLd<df, double> {
  __device__ static __forceinline__ df ld(const double* p, int i) { return df_from_double(p[i]); }
};
template <> struct SmemLd<df, float2> {
  __device__ static __forceinline__ df ld(const float2* p, int i) { float2 v = p[i]; return df{v.x, v.y}; }
};
template <> struct SmemLd<float, double> {
  __device__ static __forceinline__ float ld(const double* p, int i) { return f32_from_double(p[i]); }
};
template <> struct SmemLd<float, float> {
  __device__ static __forceinline__ float ld(const float* p, int i) { return p[i]; }
};

// base offsets (in reals) of global line g of the launch
__device__ __forceinline__ long long line_base(const LineArgs& a, unsigned g, bool out) {
  unsigned plane = a.fd_lpp.div(g);
  unsigned r = g - plane * (unsigned)a.lines_per_plane;
  unsigned c = a.fd_parts.div(r), part = r - c * (unsigned)a.parts;
  return out ? (long long)plane * a.out_plane + (long long)c * a.out_line + part
             : (long long)plane * a.in_plane + (long long)c * a.in_line + part;
}

// (line, k) of flat item t: x lines walk along a line (k fastest), y lines across lines.
template <bool OY>
__device__ __forceinline__ void split_idx(unsigned t, const FastDiv& fd_lpc, const FastDiv& fd_k, int& L, int& k) {
  if (OY) { unsigned q = fd_lpc.div(t); L = (int)(t - q * fd_lpc.d); k = (int)q; }
  else { unsigned q = fd_k.div(t); L = (int)q; k = (int)(t - q * fd_k.d); }
}

// Issue the copies of one tile into `raw` (the caller commits the group).  Returns the number
// of lines of the tile and their first global line index.
template <class SI, bool OY, int CH>
__device__ __forceinline__ int stage_tile(const LineArgs& a, int tile, SI* raw, int& gline0) {
  const SI* in = reinterpret_cast<const SI*>(a.in);
  constexpr int ES = (int)sizeof(SI);
  if (!OY) {
    const int line0 = tile * a.lpc;
    const int nl = min(a.lpc, a.nlines - line0);
    gline0 = line0;
    // rows are contiguous: one run of nl rows of in_line reals
    const unsigned char* src = reinterpret_cast<const unsigned char*>(in + line_base(a, (unsigned)line0, false));
    unsigned char* dst = reinterpret_cast<unsigned char*>(raw);
    const int bytes = nl * a.in_line * ES;
    for (int i = threadIdx.x * CH; i < bytes; i += blockDim.x * CH) cp_async<CH>(dst + i, src + i);
    return nl;
  }
  // y: tile = (plane, block of tx columns); staged as in_rows rows of raw_row reals
  const int plane = (int)a.fd_nblk.div((unsigned)tile);
  const int blk = tile - plane * a.nblk;
  const int c0 = blk * a.tx;
  const int ncols = min(a.tx, a.ncols - c0);
  gline0 = plane * a.lines_per_plane + c0 * a.parts;
  const SI* gbase = in + (long long)plane * a.in_plane + (long long)c0 * a.in_line;
  const int nrows = a.in_rows;
  if (ncols == a.tx) {
    const int cpr = (int)a.fd_cpr.d;  // chunks of CH bytes per row (tx * in_line * ES / CH, exact)
    const int tot = cpr * nrows;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      int j = (int)a.fd_cpr.div((unsigned)t), c = t - j * cpr;
      const unsigned char* src = reinterpret_cast<const unsigned char*>(gbase + (long long)j * a.in_pos) + c * CH;
      unsigned char* dst = reinterpret_cast<unsigned char*>(raw + j * a.raw_row) + c * CH;
      cp_async<CH>(dst, src);
    }
  } else {
    // ragged last column block: element-sized copies
    constexpr int EC = ES >= 8 ? 8 : 4;
    const int epr = ncols * a.in_line;  // elements per row
    const int tot = epr * nrows;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      int j = t / epr, c = t - j * epr;
      cp_async<EC>(raw + j * a.raw_row + c, gbase + (long long)j * a.in_pos + c);
    }
  }
  return ncols * a.parts;
}


// Input of one tile: either the staged copy in shared memory or the global array itself.
template <class R, class SI, bool OY> struct SrcStaged {
  const SI* raw;
  int rpos, in_line, parts;
  __device__ __forceinline__ int base(int L) const {
    if (!OY) return L * in_line;
    int c = L, part = 0;
    if (parts == 2) { c = L >> 1; part = L & 1; }
    return c * in_line + part;
  }
  __device__ __forceinline__ R ld(int b, int j) const { return SmemLd<R, SI>::ld(raw, b + j * rpos); }
};
template <class R, class SI> struct SrcGlobal {
  const SI* in;
  const long long* bases;  // per-line bases (shared memory)
  long long pos;
  __device__ __forceinline__ long long base(int L) const { return bases[L]; }
  __device__ __forceinline__ R ld(long long b, int j) const { return Io<R, SI>::ld(in, b + (long long)j * pos); }
};

// Pre-processing of one tile: builds the complex FFT input of every line in `buf`.
template <class R, bool OY, class Src>
__device__ __noinline__ void pre_tile(const LineArgs& a, const Src src, int nl, cx<R>* buf) {
  const int M = a.fp.M, N = a.N, ldm = a.ldm, kind = a.kind, nth = blockDim.x;
  const cx<R>* aux = reinterpret_cast<const cx<R>*>(a.aux);
  auto ldr = [&](auto b, int j) -> R { return src.ld(b, j); };
  auto ldc = [&](auto b, int j) -> cx<R> { return cx<R>{src.ld(b, j), src.ld(b + 1, j)}; };
    // -------------------------------------------------------------- pre-processing
    {
      const int tot = (OY ? a.lpc : nl) * M;
      for (int t = threadIdx.x; t < tot; t += nth) {
        int L, k;
        split_idx<OY>((unsigned)t, a.fd_lpc, a.fd_kpre, L, k);
        if (OY && L >= nl) continue;
        const auto b = src.base(L);
        cx<R> z;
        switch (kind) {
          case LK_R2C: z = cx<R>{ldr(b, 2 * k), ldr(b, 2 * k + 1)}; break;
          case LK_DCT2:
          case LK_DST2: {
            // v_j = u_{2j} (j < M), u_{2N-1-2j} (j >= M); DST-II alternates the sign of odd samples
            int j0 = 2 * k, j1 = 2 * k + 1;
            int s0 = j0 < M ? 2 * j0 : 2 * N - 1 - 2 * j0;
            int s1 = j1 < M ? 2 * j1 : 2 * N - 1 - 2 * j1;
            R v0 = ldr(b, s0), v1 = ldr(b, s1);
            if (kind == LK_DST2) {
              if (j0 >= M) v0 = Ar<R>::neg(v0);
              if (j1 >= M) v1 = Ar<R>::neg(v1);
            }
            z = cx<R>{v0, v1};
            break;
          }
          case LK_DCT4:
          case LK_DST4: {
            R e = ldr(b, 2 * k), o = ldr(b, N - 1 - 2 * k);
            z = (kind == LK_DCT4) ? cx<R>{e, o} : cx<R>{o, e};
            z = cmul(z, aux[k]);  // exp(-i pi (4k+1) / 4N)
            break;
          }
          case LK_C2C_F:
          case LK_C2C_I: z = ldc(b, k); break;
          case LK_C2R:
          case LK_DCT3:
          case LK_DST3: {
            // Hermitian pair (X_k, X_{M-k}) -> Z_k = E + i O, E = X_k + conj X_{M-k},
            // O = (X_k - conj X_{M-k}) exp(+2 pi i k / N); imaginary parts of X_0, X_M dropped.
            cx<R> Xk, Xm;
            if (kind == LK_C2R) {
              Xk = ldc(b, k);
              Xm = ldc(b, M - k);
            } else {
              // V_j = exp(+i pi j / 2N) (Y_j - i Y_{N-j}), Y_N = 0;  DST-III reads Y reversed
              const cx<R>* w4 = aux + (M + 1);
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
            z = cx<R>{Ar<R>::sub(E.re, O.im), Ar<R>::add(E.im, O.re)};
            break;
          }
          default: z = cx<R>{Ar<R>::zero(), Ar<R>::zero()};
        }
        buf[L * ldm + k] = z;
      }
    }

}

// Post-processing of one transformed tile: extracts the wanted transform from `buf` and writes
// it to global memory (line bases in s_bout).
template <class R, class SO, bool OY>
__device__ __noinline__ void post_tile(const LineArgs& a, const cx<R>* buf, int nl, const long long* s_bout) {
  const int M = a.fp.M, N = a.N, ldm = a.ldm, kind = a.kind, nth = blockDim.x;
  const cx<R>* aux = reinterpret_cast<const cx<R>*>(a.aux);
  SO* out = reinterpret_cast<SO*>(a.out);
  const long long op = a.out_pos;
  auto str = [&](long long b, int j, R v) { Io<R, SO>::st(out, b + (long long)j * op, v); };
  auto stc = [&](long long b, int j, cx<R> v) {
    long long o = b + (long long)j * op;
    Io<R, SO>::st(out, o, v.re);
    Io<R, SO>::st(out, o + 1, v.im);
  };
    // -------------------------------------------------------------- post-processing
    {
      const int K = (int)a.fd_kpost.d;
      const int tot = (OY ? a.lpc : nl) * K;
      for (int t = threadIdx.x; t < tot; t += nth) {
        int L, k;
        split_idx<OY>((unsigned)t, a.fd_lpc, a.fd_kpost, L, k);
        if (OY && L >= nl) continue;
        long long b = s_bout[L];
        const cx<R>* zl = buf + L * ldm;
        switch (kind) {
          case LK_R2C:
          case LK_DCT2:
          case LK_DST2: {
            cx<R> Zk = zl[k == M ? 0 : k];
            cx<R> Zm = zl[k == 0 ? 0 : M - k];
            cx<R> Zc = cconj(Zm);
            cx<R> E = chalf(cadd(Zk, Zc));
            cx<R> dd = csub(Zk, Zc);
            cx<R> O = chalf(cx<R>{dd.im, Ar<R>::neg(dd.re)});  // (Zk - conj Zm) / (2i)
            cx<R> X = cadd(E, cmul(O, aux[k]));               // + w_N^k O
            if (kind == LK_R2C) { stc(b, k, X); break; }
            cx<R> W = cmul(X, aux[M + 1 + k]);                 // exp(-i pi k / 2N)
            int i0 = k, i1 = N - k;
            if (kind == LK_DST2) { i0 = N - 1 - k; i1 = k - 1; }
            str(b, i0, W.re);
            if (k >= 1 && k < M) str(b, i1, Ar<R>::neg(W.im));
            break;
          }
          case LK_DCT4:
          case LK_DST4: {
            cx<R> s = cmul(zl[k], aux[M + k]);  // exp(-i pi k / N)
            str(b, 2 * k, s.re);
            str(b, N - 1 - 2 * k, kind == LK_DCT4 ? Ar<R>::neg(s.im) : s.im);
            break;
          }
          case LK_C2C_F:
          case LK_C2C_I: stc(b, k, zl[k]); break;
          case LK_C2R: {
            cx<R> z = zl[k];
            str(b, 2 * k, z.re);
            str(b, 2 * k + 1, z.im);
            break;
          }
          case LK_DCT3:
          case LK_DST3: {
            cx<R> z = zl[k];
            int j0 = 2 * k, j1 = 2 * k + 1;
            int s0 = j0 < M ? 2 * j0 : 2 * N - 1 - 2 * j0;
            int s1 = j1 < M ? 2 * j1 : 2 * N - 1 - 2 * j1;
            R v0 = z.re, v1 = z.im;
            if (kind == LK_DST3) {
              if (j0 >= M) v0 = Ar<R>::neg(v0);
              if (j1 >= M) v1 = Ar<R>::neg(v1);
            }
            str(b, s0, v0);
            str(b, s1, v1);
            break;
          }
          default: break;
        }
      }
    }
}

// double-float kernels need more than 128 registers per thread: they run at most 256 threads
template <class R> struct MaxThreads { static constexpr int v = std::is_same<R, df>::value ? 256 : 512; };

template <class R, class SI, class SO, bool OY, int CH>
__global__ void __launch_bounds__(MaxThreads<R>::v, 1) k_lines(const LineArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_bout[kMaxLpc];
  const LineArgs& a = args;
  const int M = a.fp.M;
  const int ldm = a.ldm;
  SI* raw0 = reinterpret_cast<SI*>(smem_raw);
  SI* raw1 = reinterpret_cast<SI*>(smem_raw + a.raw_bytes);
  cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw + 2 * (size_t)a.raw_bytes);
  cx<R>* tws = buf + (size_t)a.lpc * ldm;
  const cx<R>* twg = reinterpret_cast<const cx<R>*>(a.tw);
  for (int i = threadIdx.x; i < M; i += blockDim.x) tws[i] = twg[i];

  const int kind = a.kind;
  const int nth = blockDim.x;
  const bool inv = (kind == LK_C2R || kind == LK_C2C_I || kind == LK_DCT3 || kind == LK_DST3);

  int tile = blockIdx.x;
  int gl_next = 0, nl_next = 0;
  if (tile < a.ntiles) nl_next = stage_tile<SI, OY, CH>(a, tile, raw0, gl_next);
  cp_async_commit();

  for (int it = 0; tile < a.ntiles; tile += gridDim.x, it++) {
    const int nl = nl_next, gline0 = gl_next;
    const SI* raw = (it & 1) ? raw1 : raw0;
    // stage the next tile into the other buffer (freed by the barrier that ended the last iteration)
    if (tile + (int)gridDim.x < a.ntiles)
      nl_next = stage_tile<SI, OY, CH>(a, tile + gridDim.x, (it & 1) ? raw0 : raw1, gl_next);
    cp_async_commit();
    for (int L = threadIdx.x; L < nl; L += nth) s_bout[L] = line_base(a, (unsigned)(gline0 + L), true);
    cp_async_wait<1>();
    __syncthreads();

    pre_tile<R, OY>(a, SrcStaged<R, SI, OY>{raw, OY ? a.raw_row : a.in_pos, a.in_line, a.parts}, nl, buf);
    __syncthreads();

    // -------------------------------------------------------------- FFT
    if (inv) fft_lines<R, true>(buf, nl, ldm, a.fp, tws);
    else fft_lines<R, false>(buf, nl, ldm, a.fp, tws);
    if (a.fp.nst == 0) __syncthreads();

    post_tile<R, SO, OY>(a, buf, nl, s_bout);
    __syncthreads();  // buf, s_bout and this iteration's staging buffer are free again
  }
  cp_async_wait<0>();
}

// Direct variant: one tile per CTA, the pre-processing reads global memory (through L1).
template <class R, class SI, class SO, bool OY>
__global__ void __launch_bounds__(MaxThreads<R>::v, 1) k_lines_direct(const LineArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_bin[kMaxLpc], s_bout[kMaxLpc];
  const LineArgs& a = args;
  const int M = a.fp.M;
  const int ldm = a.ldm;
  cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tws = buf + (size_t)a.lpc * ldm;
  const cx<R>* twg = reinterpret_cast<const cx<R>*>(a.tw);
  for (int i = threadIdx.x; i < M; i += blockDim.x) tws[i] = twg[i];
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
  pre_tile<R, OY>(a, SrcGlobal<R, SI>{reinterpret_cast<const SI*>(a.in), s_bin, (long long)a.in_pos}, nl, buf);
  __syncthreads();
  if (inv) fft_lines<R, true>(buf, nl, ldm, a.fp, tws);
  else fft_lines<R, false>(buf, nl, ldm, a.fp, tws);
  if (a.fp.nst == 0) __syncthreads();
  post_tile<R, SO, OY>(a, buf, nl, s_bout);
}

// ------------------------------------------------------------------ launcher
static int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// resident CTAs per SM of one kernel configuration (cached: the launch shapes of a plan repeat)
static int blocks_per_sm(const void* fn, int threads, size_t smem) {
  struct Ent { const void* fn; int threads; size_t smem; int bpsm; };
  static std::mutex mu;
  static std::vector<Ent> cache;
  std::lock_guard<std::mutex> lk(mu);
  for (const Ent& e : cache)
    if (e.fn == fn && e.threads == threads && e.smem == smem) return e.bpsm;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem) != cudaSuccess || b < 1) b = 1;
  cache.push_back(Ent{fn, threads, smem, b});
  return b;
}

template <class R, class SI, class SO, bool OY, int CH>
static cudaError_t launch_k(const LineArgs& a, int threads, size_t smem, int grid, cudaStream_t st) {
  auto k = k_lines<R, SI, SO, OY, CH>;
  // dynamic shared memory above 48 KB must be opted into; plans keep it <= 200 KB, and the
  // kernel's static shared memory (per-line output bases) comes on top of it.
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 216 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // persistent grid: as many CTAs as can be resident, each walking over tiles
  if (grid <= 0) grid = std::min(a.ntiles, blocks_per_sm((const void*)k, threads, smem) * num_sms());
  if (grid < 1) grid = 1;
  k<<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <class R, class SI, class SO, bool OY>
static cudaError_t launch_t(const LineArgs& a, int threads, size_t smem, int grid, cudaStream_t st) {
  constexpr int ES = sizeof(SI) >= 8 ? 8 : 4;
  if (!a.staged) {
    auto k = k_lines_direct<R, SI, SO, OY>;
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 216 * 1024);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    size_t sm = (size_t)a.lpc * a.ldm * sizeof(cx<R>) + (size_t)a.fp.M * sizeof(cx<R>);
    k<<<a.ntiles, threads, sm, st>>>(a);
    return cudaGetLastError();
  }
  if (a.chunk == 16) return launch_k<R, SI, SO, OY, 16>(a, threads, smem, grid, st);
  return launch_k<R, SI, SO, OY, ES>(a, threads, smem, grid, st);
}

// storage codes
enum { ST_F64 = 0, ST_F32 = 1, ST_SPILL = 2 };

template <class R, class SP>
static cudaError_t dispatch(const LineArgs& a, int oy, int sin, int sout, int threads, size_t smem, int grid,
                            cudaStream_t st) {
  if (oy) {
    if (sin == ST_SPILL && sout == ST_SPILL) return launch_t<R, SP, SP, true>(a, threads, smem, grid, st);
    return cudaErrorInvalidValue;
  }
  if (sin == ST_F64 && sout == ST_SPILL) return launch_t<R, double, SP, false>(a, threads, smem, grid, st);
  if (sin == ST_SPILL && sout == ST_F64) return launch_t<R, SP, double, false>(a, threads, smem, grid, st);
  if (sin == ST_SPILL && sout == ST_SPILL) return launch_t<R, SP, SP, false>(a, threads, smem, grid, st);
  if (std::is_same<R, float>::value) {
    // FP32 I/O: the spill type is float as well
    if (sin == ST_F32 && sout == ST_SPILL) return launch_t<R, SP, SP, false>(a, threads, smem, grid, st);
    if (sin == ST_SPILL && sout == ST_F32) return launch_t<R, SP, SP, false>(a, threads, smem, grid, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_lines_impl(const LineArgs& a, bool df_arith, int oy, int sin, int sout, int threads, size_t smem,
                              int grid, cudaStream_t st) {
  if (df_arith) return dispatch<df, float2>(a, oy, sin, sout, threads, smem, grid, st);
  return dispatch<float, float>(a, oy, sin, sout, threads, smem, grid, st);
}

}  // namespace pp
