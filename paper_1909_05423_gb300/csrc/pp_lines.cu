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
// One CTA transforms `lpc` lines held in shared memory.  For x lines consecutive threads walk
// along a line (coalesced); for y lines consecutive threads walk across columns at a fixed
// position (coalesced rows of 16-32 values).
#include <type_traits>

#include "pp_internal.h"

namespace pp {

struct LineCtx {
  const LineArgs* a;
  int line0;
  __device__ __forceinline__ long long base_in(int L) const {
    long long g = line0 + L;
    long long plane = g / a->lines_per_plane;
    int r = (int)(g - plane * a->lines_per_plane);
    int c = r / a->parts, part = r - c * a->parts;
    return plane * a->in_plane + (long long)c * a->in_line + part;
  }
  __device__ __forceinline__ long long base_out(int L) const {
    long long g = line0 + L;
    long long plane = g / a->lines_per_plane;
    int r = (int)(g - plane * a->lines_per_plane);
    int c = r / a->parts, part = r - c * a->parts;
    return plane * a->out_plane + (long long)c * a->out_line + part;
  }
};

template <bool OY> __device__ __forceinline__ void split_idx(int t, int nl, int K, int& L, int& k) {
  if (OY) { L = t % nl; k = t / nl; }
  else { L = t / K; k = t - L * K; }
}

template <class R, class SI, class SO, bool OY>
__global__ void __launch_bounds__(512, 1) k_lines(const LineArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const LineArgs& a = args;
  const int M = a.fp.M;
  const int N = a.N;
  const int ldm = a.ldm;
  cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tws = buf + (size_t)a.lpc * ldm;
  const cx<R>* twg = reinterpret_cast<const cx<R>*>(a.tw);
  const cx<R>* aux = reinterpret_cast<const cx<R>*>(a.aux);
  for (int i = threadIdx.x; i < M; i += blockDim.x) tws[i] = twg[i];

  LineCtx ctx{&a, (int)blockIdx.x * a.lpc};
  const int nl = min(a.lpc, a.nlines - ctx.line0);
  const SI* in = reinterpret_cast<const SI*>(a.in);
  SO* out = reinterpret_cast<SO*>(a.out);
  const long long ip = a.in_pos, op = a.out_pos;
  const int kind = a.kind;
  const int nth = blockDim.x;

  auto ldr = [&](long long b, int j) -> R { return Io<R, SI>::ld(in, b + (long long)j * ip); };
  auto ldc = [&](long long b, int j) -> cx<R> {
    long long o = b + (long long)j * ip;
    return cx<R>{Io<R, SI>::ld(in, o), Io<R, SI>::ld(in, o + 1)};
  };
  auto str = [&](long long b, int j, R v) { Io<R, SO>::st(out, b + (long long)j * op, v); };
  auto stc = [&](long long b, int j, cx<R> v) {
    long long o = b + (long long)j * op;
    Io<R, SO>::st(out, o, v.re);
    Io<R, SO>::st(out, o + 1, v.im);
  };

  // ------------------------------------------------------------------ pre-processing
  {
    const int K = M;
    const int tot = nl * K;
    for (int t = threadIdx.x; t < tot; t += nth) {
      int L, k;
      split_idx<OY>(t, nl, K, L, k);
      long long b = ctx.base_in(L);
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
  __syncthreads();

  // ------------------------------------------------------------------ FFT
  const bool inv = (kind == LK_C2R || kind == LK_C2C_I || kind == LK_DCT3 || kind == LK_DST3);
  if (inv) fft_lines<R, true>(buf, nl, ldm, a.fp, tws);
  else fft_lines<R, false>(buf, nl, ldm, a.fp, tws);
  // (fft_lines ends with a barrier)
  if (a.fp.nst == 0) __syncthreads();

  // ------------------------------------------------------------------ post-processing
  {
    int K;
    switch (kind) {
      case LK_R2C:
      case LK_DCT2:
      case LK_DST2: K = M + 1; break;
      case LK_C2C_F:
      case LK_C2C_I: K = N; break;
      default: K = M;
    }
    const int tot = nl * K;
    for (int t = threadIdx.x; t < tot; t += nth) {
      int L, k;
      split_idx<OY>(t, nl, K, L, k);
      long long b = ctx.base_out(L);
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

// ------------------------------------------------------------------ launcher
template <class R, class SI, class SO, bool OY>
static cudaError_t launch_t(const LineArgs& a, int threads, size_t smem, cudaStream_t st) {
  auto k = k_lines<R, SI, SO, OY>;
  static bool attr_done = false;  // per instantiation
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  int grid = (a.nlines + a.lpc - 1) / a.lpc;
  k<<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

// storage codes
enum { ST_F64 = 0, ST_F32 = 1, ST_SPILL = 2 };

template <class R, class SP>
static cudaError_t dispatch(const LineArgs& a, int oy, int sin, int sout, int threads, size_t smem, cudaStream_t st) {
  if (oy) {
    if (sin == ST_SPILL && sout == ST_SPILL) return launch_t<R, SP, SP, true>(a, threads, smem, st);
    return cudaErrorInvalidValue;
  }
  if (sin == ST_F64 && sout == ST_SPILL) return launch_t<R, double, SP, false>(a, threads, smem, st);
  if (sin == ST_SPILL && sout == ST_F64) return launch_t<R, SP, double, false>(a, threads, smem, st);
  if (sin == ST_SPILL && sout == ST_SPILL) return launch_t<R, SP, SP, false>(a, threads, smem, st);
  if (std::is_same<R, float>::value) {
    // FP32 I/O: the spill type is float as well
    if (sin == ST_F32 && sout == ST_SPILL) return launch_t<R, SP, SP, false>(a, threads, smem, st);
    if (sin == ST_SPILL && sout == ST_F32) return launch_t<R, SP, SP, false>(a, threads, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_lines_impl(const LineArgs& a, bool df_arith, int oy, int sin, int sout, int threads, size_t smem,
                              cudaStream_t st) {
  if (df_arith) return dispatch<df, float2>(a, oy, sin, sout, threads, smem, st);
  return dispatch<float, float>(a, oy, sin, sout, threads, smem, st);
}

}  // namespace pp
