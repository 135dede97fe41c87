// pp_plan.cu -- plan creation, coefficient tables, launch sequences and the C ABI.
//
// A plan fixes the grid, the per-face boundary conditions, the spacings and the arithmetic
// mode, and precomputes on the host, in FP64:
//   * the FFT twiddles (w_M^j, or per stage in butterfly order for the compile-time lengths) and
//     the pre/post twiddles of the DCT/DST recipes (angles reduced exactly in integers, then split
//     into double-float pairs);
//   * for every (kx,ky) pair the eigenvalue shift of Table "Eigenvalues"
//     (lambda = -2 + 2 cos(theta) per axis, divided by h^2, summed over x and y) and the
//     Thomas multipliers of its z system, evaluated with the same FP64 operations as a
//     textbook Thomas elimination, truncated once they reach their fixed point.
// A solve is then five launches on the caller's stream:
//   x-forward -> y-forward -> z tridiagonal -> y-inverse -> x-inverse.
// Launch shapes (threads and lines per CTA) are chosen per line kernel and direction, by a
// heuristic or by timing candidates (autotune()).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "pp_internal.h"

namespace pp {
// the kernel family and instantiation for the launch (pp_lines.cu): double-float or FP32 arithmetic,
// x (oy = 0) or y (oy = 1) lines, storage codes of input and output
cudaError_t launch_lines_impl(const LineArgs& a, bool df_arith, int oy, int sin, int sout, int threads,
                              cudaStream_t st);
cudaError_t launch_zsolve_impl(const ZArgs& a, bool df_spill, bool zper, cudaStream_t st);
cudaError_t launch_zpart_impl(const ZArgs& a, bool df_spill, int M, cudaStream_t st);
cudaError_t launch_zdiag_impl(const ZDiagArgs& a, bool df_spill, cudaStream_t st);
}  // namespace pp

using namespace pp;

static thread_local std::string g_err;

static pp_status fail(pp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

namespace pp {
pp_status set_last_error(pp_status s, const char* msg) { return fail(s, "%s", msg); }
}  // namespace pp

#define CUDA_OK(call)                                                                      \
  do {                                                                                     \
    cudaError_t _e = (call);                                                               \
    if (_e != cudaSuccess) return fail(PP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
  } while (0)

// ------------------------------------------------------------------ fault injection
// Host-side fault injection for tests: PP_FAULT_INJECT names one failure point ("alloc": the
// plan's device allocations fail; "graph": instantiating a batch graph fails).  The failure is
// reported exactly as a real one would be; nothing reaches the GPU.
static bool inject(const char* point) {
  const char* v = getenv("PP_FAULT_INJECT");
  return v && strcmp(v, point) == 0;
}

// ------------------------------------------------------------------ helpers
// n has no prime factor above 7 (the FFT radices are 2, 3, 4, 5, 7, 8)
static bool smooth2357(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

static FftPlan make_fft(int M) {
  FftPlan f;
  f.M = M;
  f.nst = 0;
  int m = M;
  while (m % 8 == 0 && f.nst < kMaxStages) { f.rad[f.nst++] = 8; m /= 8; }
  while (m % 4 == 0 && f.nst < kMaxStages) { f.rad[f.nst++] = 4; m /= 4; }
  while (m % 2 == 0 && f.nst < kMaxStages) { f.rad[f.nst++] = 2; m /= 2; }
  while (m % 3 == 0 && f.nst < kMaxStages) { f.rad[f.nst++] = 3; m /= 3; }
  while (m % 5 == 0 && f.nst < kMaxStages) { f.rad[f.nst++] = 5; m /= 5; }
  while (m % 7 == 0 && f.nst < kMaxStages) { f.rad[f.nst++] = 7; m /= 7; }
  int s = 1;
  for (int i = 0; i < f.nst; i++) {
    f.nbl[i] = FastDiv::make((unsigned)(M / f.rad[i]));
    f.s[i] = FastDiv::make((unsigned)s);
    s *= f.rad[i];
  }
  return f;
}

// exp(-2 pi i num/den) with the angle reduced exactly: num/den = q/4 + t, |t| <= 1/8.
static void expi(long long num, long long den, double& re, double& im) {
  const double PI = 3.14159265358979323846;
  long long r = num % den;
  if (r < 0) r += den;
  // quadrant index qd = round(4 r / den), remainder a/(4 den) with |a| <= den/2
  long long qd = (4 * r + den / 2) / den;  // 0..4
  long long a = 4 * r - qd * den;          // angle = 2 pi (qd/4 + a/(4 den))
  double t = 2.0 * PI * (double)a / (4.0 * (double)den);
  double c = std::cos(t), s = std::sin(t);
  double cr, sr;  // cos, sin of the full angle
  switch (qd & 3) {
    case 0: cr = c; sr = s; break;
    case 1: cr = -s; sr = c; break;
    case 2: cr = -c; sr = -s; break;
    default: cr = s; sr = -c; break;
  }
  re = cr;
  im = -sr;
}

// Per-axis eigenvalue (unit spacing), Table "Eigenvalues"; mixed D/N axis: -2 + 2cos(pi(k+1/2)/n).
static double axis_eig(int kind, int N, int k) {
  const double PI = 3.14159265358979323846;
  switch (kind) {
    case AX_P: return -2.0 + 2.0 * cos(2.0 * PI * (double)k / N);
    case AX_NN: return -2.0 + 2.0 * cos(PI * (double)k / N);
    case AX_DD: return -2.0 + 2.0 * cos(PI * (double)(k + 1) / N);
    default: return -2.0 + 2.0 * cos(PI * (2.0 * k + 1.0) / (2.0 * N));
  }
}

static int axis_kind(int lo, int hi) {
  if (lo == PP_BC_PERIODIC || hi == PP_BC_PERIODIC) return (lo == PP_BC_PERIODIC && hi == PP_BC_PERIODIC) ? AX_P : -1;
  if (lo == PP_BC_NEUMANN && hi == PP_BC_NEUMANN) return AX_NN;
  if (lo == PP_BC_DIRICHLET && hi == PP_BC_DIRICHLET) return AX_DD;
  if (lo == PP_BC_DIRICHLET && hi == PP_BC_NEUMANN) return AX_DN;
  return AX_ND;
}

static int fwd_kind(int ax, bool complex_data) {
  switch (ax) {
    case AX_P: return complex_data ? LK_C2C_F : LK_R2C;
    case AX_NN: return LK_DCT2;
    case AX_DD: return LK_DST2;
    case AX_DN: return LK_DST4;
    default: return LK_DCT4;
  }
}
static int inv_kind(int ax, bool complex_data) {
  switch (ax) {
    case AX_P: return complex_data ? LK_C2C_I : LK_C2R;
    case AX_NN: return LK_DCT3;
    case AX_DD: return LK_DST3;
    case AX_DN: return LK_DST4;
    default: return LK_DCT4;
  }
}
// constant inverse weight of an axis (the syntheses are unnormalised)
static double axis_weight(int ax, int N) { return (ax == AX_DN || ax == AX_ND) ? 2.0 / N : 1.0 / N; }

static void split2(double v, float* o) {
  float h = (float)v;
  o[0] = h;
  o[1] = (float)(v - (double)h);
}

// Build a complex table in the plan's arithmetic type: df -> 4 floats, float -> 2 floats.
struct Tab {
  std::vector<float> v;
  bool dfm;
  void push(double re, double im) {
    if (dfm) {
      float a[2], b[2];
      split2(re, a);
      split2(im, b);
      v.push_back(a[0]); v.push_back(a[1]); v.push_back(b[0]); v.push_back(b[1]);
    } else {
      v.push_back((float)re);
      v.push_back((float)im);
    }
  }
};

static pp_status upload(void** dptr, const std::vector<float>& v) {
  size_t bytes = std::max<size_t>(v.size(), 4) * sizeof(float);
  if (inject("alloc")) return fail(PP_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu): injected failure", bytes);
  cudaError_t e = cudaMalloc(dptr, bytes);
  if (e != cudaSuccess) return fail(PP_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  if (!v.empty()) CUDA_OK(cudaMemcpy(*dptr, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice));
  return PP_OK;
}

// twiddles of one axis: stage table (M entries) and aux table for its transform family
static pp_status axis_tables(pp_plan* p, int ax, int N, bool complex_data, FftPlan& fp, void** dtw, void** daux) {
  bool dfm = (p->dtype == PP_F64);
  int M = (ax == AX_P && complex_data) ? N : N / 2;
  fp = make_fft(M);
  Tab tw{{}, dfm}, aux{{}, dfm};
  double re, im;
  if (ct_length(M)) {
    // per-stage table in butterfly order: stage (stride S, radix r), p < M/(S r), t = 1..r-1 holds
    // w_M^(p S t); the last stage has no twiddles (the sizes telescope to M - 1 entries at most)
    int S = 1;
    for (int st = 0; st < fp.nst; st++) {
      const int r = fp.rad[st];
      if (S * r < M)
        for (int p = 0; p < M / (S * r); p++)
          for (int t = 1; t < r; t++) { expi((long long)p * S * t, M, re, im); tw.push(re, im); }
      S *= r;
    }
    while ((int)(tw.v.size() / (dfm ? 4 : 2)) < M) tw.push(0.0, 0.0);  // the kernels copy M entries
  } else {
    for (int j = 0; j < M; j++) { expi(j, M, re, im); tw.push(re, im); }
  }
  if (ax == AX_P && !complex_data) {
    for (int k = 0; k <= M; k++) { expi(k, N, re, im); aux.push(re, im); }
  } else if (ax == AX_NN || ax == AX_DD) {
    for (int k = 0; k <= M; k++) { expi(k, N, re, im); aux.push(re, im); }
    for (int k = 0; k <= M; k++) { expi(k, 4LL * N, re, im); aux.push(re, im); }
  } else if (ax == AX_DN || ax == AX_ND) {
    for (int n = 0; n < M; n++) { expi(4LL * n + 1, 8LL * N, re, im); aux.push(re, im); }
    for (int k = 0; k < M; k++) { expi(k, 2LL * N, re, im); aux.push(re, im); }
  }
  pp_status s = upload(dtw, tw.v);
  if (s != PP_OK) return s;
  return upload(daux, aux.v);
}

// Thomas multipliers of one z system, w_k = h2 / m_k with m_0 = b_0, m_k = b_k - h2 w_{k-1}
// (textbook elimination with sub = super = h2), truncated at the fixed point.
struct WSeq {
  std::vector<double> pre;  // w_0 .. w_{len-1}
  double winf, wlast;
};
static void thomas_multipliers(int n, double h2, double b_first, double b_int, double b_last, WSeq& s) {
  s.pre.clear();
  if (n == 1) { s.wlast = h2 / b_first; s.winf = s.wlast; return; }
  double w = h2 / b_first;
  s.pre.push_back(w);
  for (int k = 1; k <= n - 2; k++) {
    double m = b_int - h2 * w;
    double wn = h2 / m;
    if (wn == w) break;  // fixed point: every later interior multiplier is the same
    s.pre.push_back(wn);
    w = wn;
  }
  s.winf = w;
  s.wlast = h2 / (b_last - h2 * w);
}

static pp_status z_tables(pp_plan* p) {
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const double h2 = 1.0 / (p->dz * p->dz);
  const int zlo = p->bc[4], zhi = p->bc[5];
  const bool zper = (zlo == PP_BC_PERIODIC);
  long long ncx, ncy;  // mode grid
  if (p->layout == 0) { ncx = nx / 2 + 1; ncy = ny; }
  else if (p->layout == 1) { ncx = nx; ncy = ny / 2 + 1; }
  else { ncx = nx; ncy = ny; }
  p->nmodes = ncx * ncy;
  std::vector<ZMode> modes((size_t)p->nmodes);
  std::vector<float> wtab, qtab;
  std::vector<double> lx(ncx), ly(ncy);
  for (long long i = 0; i < ncx; i++) lx[i] = axis_eig(p->kx, nx, (int)i) / (p->dx * p->dx);
  for (long long j = 0; j < ncy; j++) ly[j] = axis_eig(p->ky, ny, (int)j) / (p->dy * p->dy);
  WSeq ws;
  std::vector<double> dp, cpv;
  for (long long j = 0; j < ncy; j++) {
    for (long long i = 0; i < ncx; i++) {
      ZMode& m = modes[(size_t)(j * ncx + i)];
      memset(&m, 0, sizeof m);
      double lam = lx[i] + ly[j];
      double b_int = -2.0 * h2 + lam;
      bool sing = p->singular && i == 0 && j == 0;
      if (sing) {
        // rows 1..n-1 with u_0 pinned: b = b_int, last row + h2 for a Neumann top face
        double b_last = zper ? b_int : b_int + h2;
        // multipliers about -k/(k+1): stored as 1 + w (pp_zmul.cuh), exact in FP64 (Sterbenz)
        m.flags = ZF_SINGULAR | ZF_NEAR1;
        m.woff = (int)(wtab.size() / 2);
        int ns = nz - 1;
        double w = 0.0;
        for (int r = 0; r < ns; r++) {
          double b = (r == ns - 1) ? b_last : b_int;
          double mm = (r == 0) ? b : b - h2 * w;
          w = h2 / mm;
          float o[2];
          split2(1.0 + w, o);
          wtab.push_back(o[0]); wtab.push_back(o[1]);
        }
        m.wlen = ns;
        continue;
      }
      double b_first, b_last;
      if (zper) {
        // Sherman-Morrison: gamma = -b_0, b'_0 = b_0 - gamma, b'_{n-1} = b_{n-1} - h2 h2 / gamma
        double gamma = -b_int;
        b_first = b_int - gamma;
        b_last = b_int - h2 * h2 / gamma;
        m.flags = ZF_PERIODIC;
        thomas_multipliers(nz, h2, b_first, b_int, b_last, ws);
        // q = h2 A'^{-1} e_0 (forward elimination of e_0 decays geometrically; truncated once below
        // 2^-64 of its first entry, 2^-16 under the double-float rounding of the terms it enters)
        dp.assign(nz, 0.0);
        cpv.assign(nz, 0.0);
        auto wk = [&](int k) { return k == nz - 1 ? ws.wlast : (k < (int)ws.pre.size() ? ws.pre[k] : ws.winf); };
        int K = nz;
        for (int k = 0; k < nz; k++) {
          // dp_k = (e0_k - h2 dp_{k-1}) / m_k,  1/m_k = w_k / h2
          double rhs = (k == 0) ? 1.0 : -h2 * dp[k - 1];
          dp[k] = rhs * wk(k) / h2;
          if (k > 0 && std::fabs(dp[k]) < 0x1p-64 * std::fabs(dp[0])) { K = k; break; }
        }
        // back substitution x_k = dp_k - cp_k x_{k+1}, cp_k = w_k
        std::vector<double> q(K);
        double x = 0.0;
        for (int k = K - 1; k >= 0; k--) {
          x = (k == nz - 1) ? dp[k] : dp[k] - wk(k) * x;
          q[k] = x;
        }
        // z = A'^{-1}(gamma e_0 + h2 e_{n-1}):  z_0 and z_{n-1}
        double inv00 = q[0];
        double inv0n = (K == nz) ? q[nz - 1] : 0.0;          // (A'^{-1})_{0,n-1}
        double invnn = ws.wlast / h2;                         // (A'^{-1})_{n-1,n-1}
        double z0 = gamma * inv00 + h2 * inv0n;
        double zn = gamma * inv0n + h2 * invnn;
        double D = 1.0 / (1.0 + z0 + h2 * zn / gamma);
        split2(gamma / h2, m.gam);
        split2(h2 / gamma, m.igam);
        split2(D, m.dsm);
        m.qoff = (int)(qtab.size() / 2);
        m.qlen = K;
        for (int k = 0; k < K; k++) {
          float o[2];
          split2(h2 * q[k], o);
          qtab.push_back(o[0]); qtab.push_back(o[1]);
        }
      } else {
        b_first = b_int + (zlo == PP_BC_NEUMANN ? h2 : -h2);
        b_last = b_int + (zhi == PP_BC_NEUMANN ? h2 : -h2);
        thomas_multipliers(nz, h2, b_first, b_int, b_last, ws);
      }
      m.woff = (int)(wtab.size() / 2);
      m.wlen = (int)ws.pre.size();
      // a weakly dominant mode, whose converged multiplier (the one of most rows, whose rounding
      // would act on every row alike) lies near -1, stores 1 + w (pp_zmul.cuh)
      const bool near1 = 1.0 + ws.winf < kNear1;
      if (near1) m.flags |= ZF_NEAR1;
      for (double w : ws.pre) {
        float o[2];
        split2(near1 ? 1.0 + w : w, o);
        wtab.push_back(o[0]); wtab.push_back(o[1]);
      }
      split2(near1 ? 1.0 + ws.winf : ws.winf, m.winf);
      split2(near1 ? 1.0 + ws.wlast : ws.wlast, m.wlast);
    }
    if (wtab.size() / 2 > 0x7fffffffULL || qtab.size() / 2 > 0x7fffffffULL)
      return fail(PP_ERR_UNSUPPORTED_SIZE, "z coefficient tables exceed 2^31 entries");
  }
  size_t mb = modes.size() * sizeof(ZMode);
  cudaError_t e = cudaMalloc((void**)&p->d_modes, mb);
  if (e != cudaSuccess) return fail(PP_ERR_OUT_OF_MEMORY, "cudaMalloc(modes): %s", cudaGetErrorString(e));
  CUDA_OK(cudaMemcpy(p->d_modes, modes.data(), mb, cudaMemcpyHostToDevice));
  pp_status s = upload((void**)&p->d_wtab, wtab);
  if (s != PP_OK) return s;
  return upload((void**)&p->d_qtab, qtab);
}

// Tables of periodic z by transform: the z-line DFT (complex, length nz), the x/y eigenvalue sum of
// the mode of every real slot of a spectral plane (padding slots: -1, never singular) and the z
// eigenvalue per kz.  Same FP64 expressions as the tridiagonal tables.
static pp_status zfft_tables(pp_plan* p) {
  pp_status s = axis_tables(p, AX_P, p->nz, true, p->fz, &p->d_tw_z, &p->d_aux_z);
  if (s != PP_OK) return s;
  const int nx = p->nx, ny = p->ny;
  long long row_reals, row_valid, rows;
  bool cplx;
  if (p->layout == 1) { row_reals = 2LL * nx; row_valid = 2LL * nx; rows = ny / 2 + 1; cplx = true; }
  else if (p->layout == 0) { row_reals = p->xrow; row_valid = nx + 2; rows = ny; cplx = true; }
  else { row_reals = p->xrow; row_valid = nx; rows = ny; cplx = false; }
  std::vector<float> lam((size_t)(2 * p->splane));
  for (long long r = 0; r < rows; r++) {
    const double ly = axis_eig(p->ky, ny, (int)r) / (p->dy * p->dy);
    for (long long c = 0; c < row_reals; c++) {
      double v = -1.0;
      if (c < row_valid) v = axis_eig(p->kx, nx, (int)(cplx ? c / 2 : c)) / (p->dx * p->dx) + ly;
      split2(v, &lam[(size_t)(2 * (r * row_reals + c))]);
    }
  }
  std::vector<float> eig((size_t)(2 * p->nz));
  for (int k = 0; k < p->nz; k++) split2(axis_eig(AX_P, p->nz, k) / (p->dz * p->dz), &eig[(size_t)(2 * k)]);
  if ((s = upload((void**)&p->d_zlam, lam)) != PP_OK) return s;
  return upload((void**)&p->d_zeig, eig);
}

static void free_plan(pp_plan* p) {
  if (!p) return;
  void* ptrs[] = {p->bufA, p->bufB, p->d_tw_x, p->d_aux_x, p->d_tw_y, p->d_aux_y, p->d_modes, p->d_wtab,
                  p->d_qtab, p->d_resid, p->d_mean, p->d_host_f, p->d_host_u, p->d_status,
                  p->d_tw_z, p->d_aux_z, p->d_zlam, p->d_zeig};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (cudaStream_t s : p->host_cs)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : p->host_ev)
    if (e) cudaEventDestroy(e);
  delete p;
}

// Complex values a thread holds per FFT stage: 16 in the y kernels of 512-point lines and the FP32
// x kernels of that length (one warp per line), 8 in the other power-of-two kernels, 6 for
// 3 x 2^k, and for run-time lengths the smallest stage capacity of the line's radices: lines per
// CTA x M must not exceed this x threads.
static int values_per_thread(const FftPlan& fp, int axis, bool df_arith) {
  if (ct_length(fp.M)) return ct_values_per_thread(fp.M, axis == 1, df_arith);
  int c = kCapPerThread;
  for (int i = 0; i < fp.nst; i++) c = std::min(c, stage_capacity(fp.rad[i]));
  return c;
}

// launch shapes: threads per CTA and lines per CTA of the x and y line kernels, per direction
// (0 forward, 1 inverse).  Shared memory per CTA = the complex work buffer + the stage twiddles +
// two 8-byte line bases per line.
static void choose_shapes(pp_plan* p, const pp_plan_options* opt) {
  size_t cs = (p->dtype == PP_F64) ? 16 : 8;          // bytes per complex in shared memory
  size_t se = p->elem;                                  // bytes per spill real
  const size_t smem_cap = 200 * 1024;
  for (int dir = 0; dir < 2; dir++) {
    // requested settings of this direction (the inverse ones default to the forward ones)
    int tx_req = opt ? opt->threads_x : 0, lx_req = opt ? opt->lines_x : 0;
    int ty_req = opt ? opt->threads_y : 0, cy_req = opt ? opt->cols_y : 0;
    if (dir == 1 && opt) {
      if (opt->threads_x_inv) tx_req = opt->threads_x_inv;
      if (opt->lines_x_inv) lx_req = opt->lines_x_inv;
      if (opt->threads_y_inv) ty_req = opt->threads_y_inv;
      if (opt->cols_y_inv) cy_req = opt->cols_y_inv;
    }
    // x lines: a staged tile holds lpc rows of the wider of (grid row, spectral row)
    {
      int M = p->fx.M;
      // a CTA must hold at least one whole line: threads * (values per thread) >= M
      const int cpt = values_per_thread(p->fx, 0, p->dtype == PP_F64);
      const int tmin = std::max(32, ((M + cpt - 1) / cpt + 31) / 32 * 32);
      int T = tx_req ? tx_req : 128;
      T = std::max(T, tmin);
      int cap = cpt * T;
      int nlines = p->ny * p->nz;
      int lpc = std::max(1, cap / std::max(M, 1));
      if (lx_req) lpc = std::min(lpc, lx_req);
      lpc = std::min(lpc, kMaxLpc);
      lpc = std::min(lpc, nlines);
      int ldm = M + (M >> 5) + 1;  // one padding slot per 32 elements (see pad() in pp_fft.cuh)
      auto need = [&](int l) { return (size_t)l * ldm * cs + (size_t)M * cs + 16 * (size_t)l; };
      while (lpc > 1 && need(lpc) > smem_cap) lpc--;
      p->threads_x[dir] = T;
      p->lpc_x[dir] = lpc;
      p->ldm_x = ldm;
    }
    // y lines: a staged tile holds up to ny rows of tx columns
    {
      int M = p->fy.M;
      bool cplx_cols = (p->layout == 0);
      int parts = (cplx_cols && p->ky != AX_P) ? 2 : 1;
      int ncols = cplx_cols ? p->nx / 2 + 1 : p->nx;
      size_t col_bytes = (cplx_cols ? 2 : 1) * se;
      // CTA size: 128 threads unless that leaves column segments below one 32-byte sector
      const int cpt = values_per_thread(p->fy, 1, p->dtype == PP_F64);
      const int tmin = std::max(32, ((M + cpt - 1) / cpt + 31) / 32 * 32);
      int T = 128;
      const int tmax = 512;
      if (ty_req) T = ty_req;
      else
        while (T < tmax && (size_t)std::max(1, (cpt * T / std::max(M, 1)) / parts) * col_bytes < 32) T *= 2;
      T = std::max(T, tmin);
      int cap = cpt * T;
      int maxlines = std::max(1, cap / std::max(M, 1));
      int cols = std::max(1, maxlines / parts);
      if (cy_req) cols = std::min(cols, cy_req);
      cols = std::min(cols, kMaxLpc / parts);
      cols = std::min(cols, ncols);
      // complex columns split into two real lines need room for both
      while (cols * parts * M > cap && T < tmax) {
        T = std::min(2 * T, tmax);
        cap = cpt * T;
      }
      int ldm = M + (M >> 5) + 1;
      auto need = [&](int c) { return (size_t)c * parts * ldm * cs + (size_t)M * cs + 16 * (size_t)c * parts; };
      while (cols > 1 && need(cols) > smem_cap) cols--;
      p->threads_y[dir] = T;
      p->lpc_y[dir] = cols * parts;
      p->ldm_y = ldm;
    }
  }
  // z lines of periodic z by transform: complex columns (one per real pair of a plane), the y
  // kernels' heuristic with the z length
  if (p->zfft_ok) {
    const int M = p->fz.M;
    const size_t col_bytes = 2 * se;
    const int cpt = values_per_thread(p->fz, 1, p->dtype == PP_F64);
    const int tmin = std::max(32, ((M + cpt - 1) / cpt + 31) / 32 * 32);
    int T = 128;
    while (T < 512 && (size_t)std::max(1, cpt * T / std::max(M, 1)) * col_bytes < 32) T *= 2;
    T = std::max(T, tmin);
    int cols = std::max(1, cpt * T / std::max(M, 1));
    cols = std::min<long long>(std::min(cols, kMaxLpc), p->splane / 2);
    const int ldm = M + (M >> 5) + 1;
    auto need = [&](int c) { return (size_t)c * ldm * cs + (size_t)M * cs + 16 * (size_t)c; };
    while (cols > 1 && need(cols) > smem_cap) cols--;
    p->threads_z = T;
    p->lpc_z = cols;
    p->ldm_z = ldm;
  }
}

// ------------------------------------------------------------------ line launches
enum { ST_F64 = 0, ST_F32 = 1, ST_SPILL = 2 };

// division helpers of one launch
static void finish_args(LineArgs& a) {
  int M = a.fp.M, N = a.N, K;
  // Hermitian-pair kinds handle k and M-k in one item, k <= M/2
  switch (a.kind) {
    case LK_R2C: case LK_DCT2: case LK_DST2: K = M / 2 + 1; break;
    case LK_C2C_F: case LK_C2C_I: K = N; break;
    default: K = M;
  }
  const bool herm_in = (a.kind == LK_C2R || a.kind == LK_DCT3 || a.kind == LK_DST3);
  a.fd_kpre = FastDiv::make((unsigned)(herm_in ? M / 2 + 1 : M));
  a.fd_kpost = FastDiv::make((unsigned)K);
  a.fd_lpc = FastDiv::make((unsigned)a.lpc);
  a.fd_lpp = FastDiv::make((unsigned)a.lines_per_plane);
  a.fd_parts = FastDiv::make((unsigned)a.parts);
}

namespace pp {
// Complex columns of the FP32 kernels (C2C y lines, z lines of the z transform): 16-byte vectors of
// VC = 2 adjacent complex lines when every group start is 16-byte aligned -- complex lines at real
// offset 2L, planes, positions and both pointers in multiples of 2 VC reals.  Scalar 4-byte accesses
// and a line index per item left the FP32 1024-point y C2C at twice the time per byte of the real
// kinds (4.60 -> 3.62 ms at 1024^3 with the vectors).  The double-float kernels keep the scalar
// path (5 % faster C2C with vectors, but 1 % slower real kinds from the larger code).
static void set_vec_complex(LineArgs& a, bool dfm, const void* in, const void* out) {
  if (dfm || (a.kind != LK_C2C_F && a.kind != LK_C2C_I)) return;
  const int VC = 2, R = 2 * VC;
  if (a.in_line == 2 && a.out_line == 2 && a.lpc % VC == 0 && a.in_plane % R == 0 && a.out_plane % R == 0 &&
      a.in_pos % R == 0 && a.out_pos % R == 0 && ((uintptr_t)in | (uintptr_t)out) % 16 == 0) {
    a.vec_y = 2;
    a.fd_gpc = FastDiv::make((unsigned)(a.lpc / VC));
  }
}

// bytes per real of a storage code
static size_t st_bytes(const pp_plan* p, int code) { return code == ST_F64 ? 8 : (code == ST_F32 ? 4 : p->elem); }

// axis 0 = x, 1 = y; dir 0 = forward, 1 = inverse.  io_in / io_out: ST_* codes.
cudaError_t launch_lines(const pp_plan* p, int axis, int dir, int io_in, int io_out, const void* in, void* out,
                         cudaStream_t st, int z0, int nzc) {
  LineArgs a;
  memset(&a, 0, sizeof a);
  if (nzc < 0) { z0 = 0; nzc = p->nz; }
  if (z0 < 0 || nzc < 1 || z0 + nzc > p->nz) return cudaErrorInvalidValue;
  const bool dfm = (p->dtype == PP_F64);
  const long long nxy = (long long)p->nx * p->ny;
  if (axis == 0) {
    bool per = (p->kx == AX_P);
    a.N = p->nx;
    a.kind = dir == 0 ? fwd_kind(p->kx, false) : inv_kind(p->kx, false);
    a.nlines = p->ny * nzc;
    a.lines_per_plane = p->ny;
    a.parts = 1;
    a.lpc = p->lpc_x[dir];
    a.ldm = p->ldm_x;
    a.fp = p->fx;
    a.tw = p->d_tw_x;
    a.aux = p->d_aux_x;
    long long grid_plane = nxy, grid_row = p->nx;
    long long sp_plane = p->xplane, sp_row = p->xrow;
    if (dir == 0) {
      a.in_plane = grid_plane; a.in_line = (int)grid_row; a.in_pos = 1;
      a.out_plane = sp_plane; a.out_line = sp_row; a.out_pos = per ? 2 : 1;
    } else {
      a.in_plane = sp_plane; a.in_line = (int)sp_row; a.in_pos = per ? 2 : 1;
      a.out_plane = grid_plane; a.out_line = grid_row; a.out_pos = 1;
    }
    // planes z0 .. z0+nzc-1
    in = static_cast<const char*>(in) + (size_t)z0 * a.in_plane * st_bytes(p, io_in);
    out = static_cast<char*>(out) + (size_t)z0 * a.out_plane * st_bytes(p, io_out);
    a.in = in;
    a.out = out;
    if ((long long)a.lpc * a.fp.M > (long long)values_per_thread(a.fp, 0, dfm) * p->threads_x[dir])
      return cudaErrorInvalidConfiguration;
    a.ntiles = (a.nlines + a.lpc - 1) / a.lpc;
    a.vec_ok = (((uintptr_t)in | (uintptr_t)out) % 32 == 0) ? 1 : 0;
    a.fd_gpc = FastDiv::make(1u);
    finish_args(a);
    return launch_lines_impl(a, dfm, 0, io_in, io_out, p->threads_x[dir], st);
  }
  // y
  const bool cplx_cols = (p->layout == 0);
  a.N = p->ny;
  a.kind = dir == 0 ? fwd_kind(p->ky, cplx_cols) : inv_kind(p->ky, cplx_cols);
  int parts = (cplx_cols && p->ky != AX_P) ? 2 : 1;
  int ncols = cplx_cols ? p->nx / 2 + 1 : p->nx;
  a.parts = parts;
  a.lines_per_plane = ncols * parts;
  a.nlines = a.lines_per_plane * nzc;
  a.lpc = p->lpc_y[dir];
  a.ldm = p->ldm_y;
  a.fp = p->fy;
  a.tw = p->d_tw_y;
  a.aux = p->d_aux_y;
  // x-spectral side: columns of the x-transformed array
  long long xs_plane = p->xplane, xs_col = cplx_cols ? 2 : 1, xs_pos = p->xrow;
  // fully spectral side
  long long s_plane = p->splane, s_col, s_pos;
  if (p->layout == 1) { s_col = 2; s_pos = 2LL * p->nx; }
  else { s_col = xs_col; s_pos = xs_pos; }
  if (dir == 0) {
    a.in_plane = xs_plane; a.in_line = (int)xs_col; a.in_pos = (int)xs_pos;
    a.out_plane = s_plane; a.out_line = s_col; a.out_pos = s_pos;
  } else {
    a.in_plane = s_plane; a.in_line = (int)s_col; a.in_pos = (int)s_pos;
    a.out_plane = xs_plane; a.out_line = xs_col; a.out_pos = xs_pos;
  }
  // planes z0 .. z0+nzc-1
  in = static_cast<const char*>(in) + (size_t)z0 * a.in_plane * st_bytes(p, io_in);
  out = static_cast<char*>(out) + (size_t)z0 * a.out_plane * st_bytes(p, io_out);
  a.in = in;
  a.out = out;
  if ((long long)a.lpc * a.fp.M > (long long)values_per_thread(a.fp, 1, dfm) * p->threads_y[dir])
    return cudaErrorInvalidConfiguration;
  a.tx = a.lpc / parts;
  a.ncols = ncols;
  a.nblk = (ncols + a.tx - 1) / a.tx;
  a.ntiles = a.nblk * nzc;
  {
    // 16-byte vectors of V adjacent real lines: the tile row must be contiguous (line L at real
    // offset L) and every vector start aligned (checked through all strides and both pointers)
    const int V = dfm ? 2 : 4;
    const bool real_lines = (a.kind == LK_DCT2 || a.kind == LK_DST2 || a.kind == LK_DCT3 || a.kind == LK_DST3 ||
                             a.kind == LK_DCT4 || a.kind == LK_DST4);
    a.vec_y = (real_lines && a.in_line == parts && a.out_line == parts && a.lpc % V == 0 && a.in_plane % V == 0 &&
               a.out_plane % V == 0 && a.in_pos % V == 0 && a.out_pos % V == 0 &&
               ((uintptr_t)in | (uintptr_t)out) % 16 == 0) ? 1 : 0;
    a.fd_gpc = FastDiv::make((unsigned)std::max(1, a.lpc / V));
    set_vec_complex(a, dfm, in, out);
  }
  finish_args(a);
  a.fd_nblk = FastDiv::make((unsigned)a.nblk);
  return launch_lines_impl(a, dfm, 1, io_in, io_out, p->threads_y[dir], st);
}

static void zsolve_args(const pp_plan* p, void* data, int transpose, ZArgs& a) {
  memset(&a, 0, sizeof a);
  a.data = data;
  a.plane = p->splane;
  a.nz = p->nz;
  a.cplx = (p->layout != 2);
  a.nreal = p->splane;
  // rows of the spectral plane: padded row length (reals) and the reals that carry modes
  if (p->layout == 1) { a.row_reals = 2 * p->nx; a.row_valid = 2 * p->nx; a.row_modes = p->nx; }
  else if (p->layout == 0) { a.row_reals = (int)p->xrow; a.row_valid = p->nx + 2; a.row_modes = p->nx / 2 + 1; }
  else { a.row_reals = (int)p->xrow; a.row_valid = p->nx; a.row_modes = p->nx; }
  a.fd_row = FastDiv::make((unsigned)a.row_reals);
  a.modes = p->d_modes;
  a.wtab = p->d_wtab;
  a.qtab = p->d_qtab;
  split2(p->zscale, a.scale);
  a.transpose = transpose;
  a.rstat = p->d_status;
  a.dmin = 0x1p-100f;
  a.umax = (float)(0x1p124 / ((double)p->nx * (double)p->ny));
  // the checkpointed double-float sweeps keep their checkpoints in the other spectral buffer, which
  // no stage reads between the y-forward (its last reader) and the y-inverse (its next writer)
  a.ck = (p->dtype == PP_F64 && data == p->bufB) ? p->bufA : nullptr;  // every pipeline solves z in bufB
}

cudaError_t launch_zsolve(const pp_plan* p, void* data, int transpose, cudaStream_t st) {
  ZArgs a;
  zsolve_args(p, data, transpose, a);
  const bool zper = p->bc[4] == PP_BC_PERIODIC;
  // the partitioned solve runs the forward factorisation of non-periodic z (the transposed one of
  // the adjoint stays on the Thomas sweeps); it leaves the singular mode to the pinned sweep
  if (p->zsplit > 1 && !zper && !transpose) {
    cudaError_t e = launch_zpart_impl(a, p->dtype == PP_F64, p->zsplit, st);
    if (e != cudaSuccess || !p->singular) return e;
    return launch_zsingular(p, data, st);
  }
  return launch_zsolve_impl(a, p->dtype == PP_F64, zper, st);
}

cudaError_t launch_zsingular(const pp_plan* p, void* data, cudaStream_t st) {
  ZArgs a;
  zsolve_args(p, data, 0, a);
  a.only_singular = 1;
  return launch_zsolve_impl(a, p->dtype == PP_F64, false, st);
}

// z lines as strided columns: the y-orientation kernels with one "plane" of splane/2 complex columns
// (adjacent columns 2 reals apart) and positions one z-plane apart; in place (a tile is read whole
// before it is written)
static cudaError_t launch_zlines(const pp_plan* p, int dir, void* data, cudaStream_t st) {
  LineArgs a;
  memset(&a, 0, sizeof a);
  const bool dfm = (p->dtype == PP_F64);
  const long long ncols = p->splane / 2;
  a.N = p->nz;
  a.kind = dir == 0 ? LK_C2C_F : LK_C2C_I;
  a.parts = 1;
  a.lines_per_plane = (int)ncols;
  a.nlines = (int)ncols;
  a.lpc = p->lpc_z;
  a.ldm = p->ldm_z;
  a.fp = p->fz;
  a.tw = p->d_tw_z;
  a.aux = p->d_aux_z;
  a.in_plane = 0; a.out_plane = 0;
  a.in_line = 2; a.out_line = 2;
  a.in_pos = (int)p->splane; a.out_pos = p->splane;
  a.in = data;
  a.out = data;
  if ((long long)a.lpc * a.fp.M > (long long)values_per_thread(a.fp, 1, dfm) * p->threads_z)
    return cudaErrorInvalidConfiguration;
  a.tx = a.lpc;
  a.ncols = (int)ncols;
  a.nblk = (int)((ncols + a.tx - 1) / a.tx);
  a.ntiles = a.nblk;
  a.vec_y = 0;
  a.fd_gpc = FastDiv::make(1u);
  set_vec_complex(a, dfm, data, data);
  finish_args(a);
  a.fd_nblk = FastDiv::make((unsigned)a.nblk);
  return launch_lines_impl(a, dfm, 1, ST_SPILL, ST_SPILL, p->threads_z, st);
}

cudaError_t launch_zfft(const pp_plan* p, void* data, cudaStream_t st) {
  cudaError_t e = launch_zlines(p, 0, data, st);
  if (e != cudaSuccess) return e;
  ZDiagArgs d;
  memset(&d, 0, sizeof d);
  d.data = data;
  d.plane = p->splane;
  d.nreal = p->splane;
  d.nz = p->nz;
  d.lam = p->d_zlam;
  d.zeig = p->d_zeig;
  split2(axis_weight(p->kx, p->nx) * axis_weight(p->ky, p->ny) / p->nz, d.scale);
  if (p->layout == 1) { d.row_reals = 2 * p->nx; d.row_valid = 2 * p->nx; }
  else if (p->layout == 0) { d.row_reals = (int)p->xrow; d.row_valid = p->nx + 2; }
  else { d.row_reals = (int)p->xrow; d.row_valid = p->nx; }
  d.fd_row = FastDiv::make((unsigned)d.row_reals);
  d.rstat = p->d_status;
  d.dmin = 0x1p-100f;
  d.umax = (float)(0x1p124 / ((double)p->nx * (double)p->ny * (double)p->nz));
  e = launch_zdiag_impl(d, p->dtype == PP_F64, st);
  if (e != cudaSuccess) return e;
  return launch_zlines(p, 1, data, st);
}
}  // namespace pp

// One stage of the pipeline; the line stages may be restricted to planes z0 .. z0+nzc-1 (nzc < 0:
// all planes; f and u always point at plane 0).
// io: storage of f and u (ST_F64 / ST_F32); -1 = the plan's I/O type.  An FP32-transform plan may
// also run with FP32 I/O (the refinement step's correction solve).
static pp_status run_stage(pp_plan* p, int stage, const void* f, void* u, int transpose, cudaStream_t st,
                           int z0 = 0, int nzc = -1, int io = -1, int io_out = -1) {
  if (io < 0) io = (p->dtype == PP_MIXED_F32IO) ? ST_F32 : ST_F64;
  if (io_out < 0) io_out = io;
  cudaError_t e = cudaSuccess;
  static const char* names[] = {"x-forward", "y-forward", "z-solve", "y-inverse", "x-inverse"};
  switch (stage) {
    case 0: e = launch_lines(p, 0, 0, io, ST_SPILL, f, p->bufA, st, z0, nzc); break;
    case 1: e = launch_lines(p, 1, 0, ST_SPILL, ST_SPILL, p->bufA, p->bufB, st, z0, nzc); break;
    case 2:
      // periodic z by transform is self-adjoint (the z eigenvalues are even in kz)
      e = (p->zmethod == ZM_FFT) ? launch_zfft(p, p->bufB, st) : launch_zsolve(p, p->bufB, transpose, st);
      break;
    case 3: e = launch_lines(p, 1, 1, ST_SPILL, ST_SPILL, p->bufB, p->bufA, st, z0, nzc); break;
    case 4: e = launch_lines(p, 0, 1, ST_SPILL, io_out, p->bufA, u, st, z0, nzc); break;
    default: return fail(PP_ERR_INVALID_ARG, "stage %d out of range", stage);
  }
  if (e != cudaSuccess) return fail(PP_ERR_CUDA, "%s launch: %s", names[stage], cudaGetErrorString(e));
  return PP_OK;
}

static pp_status run_pipeline(pp_plan* p, const void* f, void* u, int transpose, cudaStream_t st, int io = -1,
                              int io_out = -1) {
  for (int s = 0; s < 5; s++) {
    pp_status r = run_stage(p, s, f, u, transpose, st, 0, -1, io, io_out);
    if (r != PP_OK) return r;
  }
  return PP_OK;
}

namespace pp {
// The refined solve on caller-provided scratch (pp_solve_refined and pp_solve_refined_noalloc):
// u0 = solve(f) with FP32 output into the first half of scratch, r = f - A u0 into the second half
// (FP32), the correction solve delta = solve(r) in place with FP32 I/O, u = u0 + delta (- mean u0
// when singular).  scratch: 2 nx*ny*nz floats; partials: kMeanParts float2; mean: one float2.
pp_status solve_refined_core(pp_plan* p, const void* f, void* u, void* scratch, void* partials, void* mean,
                             cudaStream_t st) {
  const size_t n = (size_t)p->nx * p->ny * p->nz;
  float* u0 = static_cast<float*>(scratch);
  float* r = u0 + n;
  pp_status s = run_pipeline(p, f, u0, 0, st, ST_F64, ST_F32);
  if (s != PP_OK) return s;
  cudaError_t e = launch_residual(p, f, u0, r, st);
  if (e != cudaSuccess) return fail(PP_ERR_CUDA, "residual launch: %s", cudaGetErrorString(e));
  s = run_pipeline(p, r, r, 0, st, ST_F32);
  if (s != PP_OK) return s;
  // A singular problem is solved for the mean-free u; the FP32 first solve leaves a constant offset
  // that the refinement step cannot see (it lies in the null space), so it is removed explicitly.
  const void* shift = nullptr;
  if (p->singular) {
    e = launch_mean(p, u0, partials, kMeanParts, mean, st);
    if (e != cudaSuccess) return fail(PP_ERR_CUDA, "mean launch: %s", cudaGetErrorString(e));
    shift = mean;
  }
  e = launch_add(p, u, u0, r, shift, st);
  if (e != cudaSuccess) return fail(PP_ERR_CUDA, "update launch: %s", cudaGetErrorString(e));
  return PP_OK;
}
}  // namespace pp

// ------------------------------------------------------------------ autotuner
// Times candidate launch shapes of each of the four line kernels on scratch grids and keeps the
// fastest.  Results are cached per (device, sizes, boundary set, dtype) for the life of the
// process.
namespace {
struct TuneEnt {
  int dev, nx, ny, nz, dtype, bc[6];
  bool zmethod_free, zsplit_free;  // the z choices below were timed (else the caller's)
  pp_plan_options best;
  int zmethod, zsplit;
};
std::mutex g_tune_mu;
std::vector<TuneEnt> g_tune_cache;
}  // namespace

static pp_status autotune(pp_plan* p, bool zmethod_free, bool zsplit_free) {
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEnt& e : g_tune_cache)
      if (e.dev == dev && e.nx == p->nx && e.ny == p->ny && e.nz == p->nz && e.dtype == p->dtype &&
          memcmp(e.bc, p->bc, sizeof e.bc) == 0 && e.zmethod_free == zmethod_free &&
          e.zsplit_free == zsplit_free) {
        choose_shapes(p, &e.best);
        if (zmethod_free) p->zmethod = e.zmethod;
        if (zsplit_free) p->zsplit = e.zsplit;
        return PP_OK;
      }
  }
  const size_t io = (p->dtype == PP_MIXED_F32IO) ? 4 : 8;
  const size_t bytes = (size_t)p->nx * p->ny * p->nz * io;
  void *f = nullptr, *u = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaMalloc(&f, bytes);
  if (ce == cudaSuccess) ce = cudaMalloc(&u, bytes);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  // timing input: non-constant normal values, so conversions and transforms take their usual paths
  if (ce == cudaSuccess) ce = launch_fill(f, (long long)p->nx * p->ny * p->nz, io == 4, st);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  auto cleanup = [&]() {
    if (f) cudaFree(f);
    if (u) cudaFree(u);
    if (st) cudaStreamDestroy(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (ce != cudaSuccess) { cleanup(); return fail(PP_ERR_OUT_OF_MEMORY, "autotune scratch: %s", cudaGetErrorString(ce)); }
  // Time one stage (3 runs after one warm-up), in ms per launch; +inf on a failed launch.  A stage
  // whose grid is too small to fill the GPU is timed as K concurrent copies on K streams (time / K):
  // its throughput when other work shares the GPU, as in a batched graph, rather than the latency
  // of a lone launch, which favours small tiles that a shared GPU does not reward.  The copies race
  // on the scratch buffers (in bounds; the values are discarded).
  constexpr int kTuneStreams = 16;
  cudaStream_t side[kTuneStreams] = {};
  cudaEvent_t sev[kTuneStreams] = {};
  bool side_ok = true;
  for (int i = 0; i < kTuneStreams && side_ok; i++)
    side_ok = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&sev[i], cudaEventDisableTiming) == cudaSuccess;
  auto stage_ctas = [&](int s0) -> long long {
    if (s0 == 0 || s0 == 4) return ((long long)p->ny * p->nz + p->lpc_x[s0 == 4] - 1) / p->lpc_x[s0 == 4];
    const int parts = (p->layout == 0 && p->ky != AX_P) ? 2 : 1;
    const long long ncols = (p->layout == 0) ? p->nx / 2 + 1 : p->nx;
    const long long tx = std::max(1, p->lpc_y[s0 == 3] / parts);
    return (ncols + tx - 1) / tx * p->nz;
  };
  int sm_count = 152;
  cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
  auto time_stage = [&](int s0) -> float {
    const long long fill = 16LL * sm_count;  // CTAs for several full waves
    int K = 1;
    if (side_ok && s0 != 2) {
      const long long c = std::max(1LL, stage_ctas(s0));
      K = (int)std::min<long long>(kTuneStreams, (fill + c - 1) / c);
    }
    float best = 1e30f;
    for (int r = 0; r < 4; r++) {
      cudaEventRecord(e0, st);
      if (K == 1) {
        if (run_stage(p, s0, f, u, 0, st) != PP_OK) return 1e30f;
      } else {
        for (int i = 0; i < K; i++) {
          cudaStreamWaitEvent(side[i], e0, 0);
          if (run_stage(p, s0, f, u, 0, side[i]) != PP_OK) return 1e30f;
          cudaEventRecord(sev[i], side[i]);
          cudaStreamWaitEvent(st, sev[i], 0);
        }
      }
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) best = std::min(best, ms / K);
    }
    return best;
  };
  const int tcand[] = {64, 128, 256, 512};
  pp_plan_options best;
  memset(&best, 0, sizeof best);
  // Each line stage is tuned on its own, in pipeline order, so that every stage reads the output
  // of the previous one: x-forward, y-forward, (z), y-inverse, x-inverse.  Candidates: CTA sizes
  // x {as many lines as fit, half of them}.
  float bt[4] = {1e30f, 1e30f, 1e30f, 1e30f};
  const int stages[4] = {0, 1, 3, 4};
  for (int si = 0; si < 4; si++) {
    const int stage = stages[si];
    const bool xa = (stage == 0 || stage == 4), inv = (stage >= 3);
    if (stage == 3 && run_stage(p, 2, f, u, 0, st) != PP_OK) break;  // z solve between the y stages
    for (int T : tcand) {
      for (int half = 0; half < 2; half++) {
        pp_plan_options o = best;
        int* tr = xa ? (inv ? &o.threads_x_inv : &o.threads_x) : (inv ? &o.threads_y_inv : &o.threads_y);
        int* lr = xa ? (inv ? &o.lines_x_inv : &o.lines_x) : (inv ? &o.cols_y_inv : &o.cols_y);
        *tr = T;
        *lr = 0;
        choose_shapes(p, &o);
        if (half) {
          const int parts = (!xa && p->layout == 0 && p->ky != AX_P) ? 2 : 1;
          const int have = (xa ? p->lpc_x[inv] : p->lpc_y[inv]) / parts;
          if (have < 2) continue;
          *lr = have / 2;
          choose_shapes(p, &o);
        }
        const float t = time_stage(stage);
        if (t < bt[si]) {
          bt[si] = t;
          const int* got = xa ? p->threads_x : p->threads_y;
          if (xa) { if (inv) { best.threads_x_inv = got[1]; best.lines_x_inv = o.lines_x_inv; } else { best.threads_x = got[0]; best.lines_x = o.lines_x; } }
          else { if (inv) { best.threads_y_inv = got[1]; best.cols_y_inv = o.cols_y_inv; } else { best.threads_y = got[0]; best.cols_y = o.cols_y; } }
        }
      }
    }
    choose_shapes(p, &best);
    if (run_stage(p, stage, f, u, 0, st) != PP_OK) break;  // leave this stage's output for the next one
  }
  const float bx = std::max(bt[0], bt[3]), by = std::max(bt[1], bt[2]);
  // periodic z: Sherman-Morrison sweeps or the z transform, unless the caller chose one
  int zbest = p->zmethod;
  if (p->zfft_ok && zmethod_free) {
    float tz[2];
    for (int m = 0; m < 2; m++) {
      p->zmethod = m;
      tz[m] = time_stage(2);
    }
    zbest = (tz[ZM_FFT] < tz[ZM_SM]) ? ZM_FFT : ZM_SM;
  }
  p->zmethod = zbest;
  // non-periodic z: the Thomas sweeps or the partitioned solve with 8 / 16 / 32 rows per chunk,
  // timed as a lone launch (the partitioned solve trades extra arithmetic for parallelism, which
  // pays when a plan has too few modes to fill the GPU)
  if (zsplit_free && p->bc[4] != PP_BC_PERIODIC) {
    int sbest = 1;
    float tbest = 1e30f;
    for (int M : {1, kZSplitRows[0], kZSplitRows[1], kZSplitRows[2]}) {
      int G, lgG, P;
      if (M > 1 && !zpart_shape(p->nz, M, &G, &lgG, &P)) continue;
      p->zsplit = M;
      const float t = time_stage(2);
      if (t < tbest) { tbest = t; sbest = M; }
    }
    p->zsplit = sbest;
  }
  cudaStreamSynchronize(st);
  for (int i = 0; i < kTuneStreams; i++) {
    if (side[i]) cudaStreamSynchronize(side[i]), cudaStreamDestroy(side[i]);
    if (sev[i]) cudaEventDestroy(sev[i]);
  }
  cleanup();
  // the timing runs' status (scratch data) is not the caller's
  cudaMemset(p->d_status, 0, sizeof(unsigned));
  if (bx >= 1e30f || by >= 1e30f) return fail(PP_ERR_CUDA, "autotune: no candidate launch shape ran");
  choose_shapes(p, &best);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  TuneEnt ent;
  ent.dev = dev; ent.nx = p->nx; ent.ny = p->ny; ent.nz = p->nz; ent.dtype = p->dtype;
  memcpy(ent.bc, p->bc, sizeof ent.bc);
  ent.zmethod_free = zmethod_free;
  ent.zsplit_free = zsplit_free;
  ent.best = best;
  ent.zmethod = p->zmethod;
  ent.zsplit = p->zsplit;
  g_tune_cache.push_back(ent);
  return PP_OK;
}

// ------------------------------------------------------------------ batched solves as one graph
// A batch (plans[i]: f[i] -> u[i]) is captured once into a CUDA graph -- the five launches of
// every member -- and replayed with a single cudaGraphLaunch while the same plans and pointers
// come back.  Destroying a plan evicts every cached graph that uses it.
namespace {
struct BatchGraph {
  std::vector<const void*> key;  // plans, then f, then u
  cudaGraphExec_t exec;
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch_cache;  // most recent last
constexpr size_t kBatchCacheMax = 8;
// Settings chosen for a list of plans (see tune_batch): 0 = every member's own, 1 = the shared-GPU
// settings for its autotuned members.  Kept while all of the plans live.
struct BatchChoice {
  std::vector<const pp_plan*> plans;
  int choice;
};
std::vector<BatchChoice> g_batch_choice;
constexpr size_t kBatchChoiceMax = 64;

void evict_plan(const pp_plan* p) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t i = 0; i < g_batch_choice.size();) {
    const auto& v = g_batch_choice[i].plans;
    if (std::find(v.begin(), v.end(), p) != v.end()) g_batch_choice.erase(g_batch_choice.begin() + i);
    else i++;
  }
  for (size_t i = 0; i < g_batch_cache.size();) {
    const auto& k = g_batch_cache[i].key;
    size_t n = k.size() / 3;
    bool uses = false;
    for (size_t j = 0; j < n; j++) uses |= (k[j] == p);
    if (uses) {
      cudaGraphExecDestroy(g_batch_cache[i].exec);
      g_batch_cache.erase(g_batch_cache.begin() + i);
    } else {
      i++;
    }
  }
}
}  // namespace

// Launch settings of a plan that a batched graph may swap: launch shapes and the z algorithm.
struct PlanSettings {
  int threads_x[2], lpc_x[2], ldm_x, threads_y[2], lpc_y[2], ldm_y, threads_z, lpc_z, ldm_z, zsplit, zmethod;
};
static PlanSettings get_settings(const pp_plan* p) {
  PlanSettings s;
  for (int d = 0; d < 2; d++) {
    s.threads_x[d] = p->threads_x[d]; s.lpc_x[d] = p->lpc_x[d];
    s.threads_y[d] = p->threads_y[d]; s.lpc_y[d] = p->lpc_y[d];
  }
  s.ldm_x = p->ldm_x; s.ldm_y = p->ldm_y;
  s.threads_z = p->threads_z; s.lpc_z = p->lpc_z; s.ldm_z = p->ldm_z;
  s.zsplit = p->zsplit;
  s.zmethod = p->zmethod;
  return s;
}
static void set_settings(pp_plan* p, const PlanSettings& s) {
  for (int d = 0; d < 2; d++) {
    p->threads_x[d] = s.threads_x[d]; p->lpc_x[d] = s.lpc_x[d];
    p->threads_y[d] = s.threads_y[d]; p->lpc_y[d] = s.lpc_y[d];
  }
  p->ldm_x = s.ldm_x; p->ldm_y = s.ldm_y;
  p->threads_z = s.threads_z; p->lpc_z = s.lpc_z; p->ldm_z = s.ldm_z;
  p->zsplit = s.zsplit;
  p->zmethod = s.zmethod;
}

// Puts the autotuned members of a batch on the library's shared-GPU settings -- the default launch
// shapes and, where the autotuner chose the z algorithm, the Thomas or Sherman-Morrison sweeps
// (the partitioned solve and the z transform buy a lone plan latency with extra work) -- for the
// scope of one capture, and restores their own settings afterwards (a captured graph keeps the
// launch parameters it was captured with).
struct SettingsSwap {
  std::vector<std::pair<pp_plan*, PlanSettings>> saved;
  void apply(pp_plan* const* plans, int n) {
    for (int i = 0; i < n; i++) {
      pp_plan* p = plans[i];
      if (!p->tuned) continue;
      bool seen = false;
      for (const auto& s : saved) seen |= (s.first == p);
      if (seen) continue;
      saved.emplace_back(p, get_settings(p));
      choose_shapes(p, nullptr);
      if (p->z_tuned) {
        p->zsplit = 1;
        p->zmethod = ZM_SM;
      }
    }
  }
  ~SettingsSwap() {
    for (const auto& s : saved) set_settings(s.first, s.second);
  }
};

// Capture the batch on private streams: a fork event fans the members out over up to
// kBranches capture streams (members that share a plan stay on one branch, in order, since
// they share its workspace), a join brings them back; the graph's branches run concurrently.
static pp_status capture_batch(pp_plan* const* plans, const void* const* f, void* const* u, int n,
                               cudaGraphExec_t* out) {
  constexpr int kBranches = 32;
  std::vector<const pp_plan*> uniq;
  std::vector<int> branch(n);
  for (int i = 0; i < n; i++) {
    int b = -1;
    for (size_t j = 0; j < uniq.size(); j++)
      if (uniq[j] == plans[i]) { b = (int)(j % kBranches); break; }
    if (b < 0) { b = (int)(uniq.size() % kBranches); uniq.push_back(plans[i]); }
    branch[i] = b;
  }
  const int nb = (int)std::min<size_t>(uniq.size(), kBranches);
  cudaStream_t cap;
  CUDA_OK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  std::vector<cudaStream_t> br(nb, nullptr);
  std::vector<cudaEvent_t> ev(nb + 1, nullptr);
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < nb && e == cudaSuccess; b++) e = cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking);
  for (int b = 0; b <= nb && e == cudaSuccess; b++) e = cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming);
  auto cleanup = [&]() {
    for (cudaStream_t x : br) if (x) cudaStreamDestroy(x);
    for (cudaEvent_t x : ev) if (x) cudaEventDestroy(x);
    cudaStreamDestroy(cap);
  };
  if (e != cudaSuccess) { cleanup(); return fail(PP_ERR_CUDA, "batch streams/events: %s", cudaGetErrorString(e)); }
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cleanup();
    return fail(PP_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
  }
  pp_status s = PP_OK;
  e = cudaEventRecord(ev[nb], cap);
  for (int b = 0; b < nb && e == cudaSuccess; b++) e = cudaStreamWaitEvent(br[b], ev[nb], 0);
  if (e != cudaSuccess) s = fail(PP_ERR_CUDA, "batch fork: %s", cudaGetErrorString(e));
  for (int i = 0; i < n && s == PP_OK; i++) s = run_pipeline(plans[i], f[i], u[i], 0, br[branch[i]]);
  for (int b = 0; b < nb; b++) {
    cudaEventRecord(ev[b], br[b]);
    cudaStreamWaitEvent(cap, ev[b], 0);
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cap, &graph);
  cleanup();
  if (s != PP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(PP_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = inject("graph") ? cudaErrorInvalidValue : cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(PP_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  *out = exec;
  return PP_OK;
}

// Shortest of three replays of an executable graph on st (after one warm-up), ms; +inf on error.
static float time_graph(cudaGraphExec_t g, cudaStream_t st) {
  cudaEvent_t a = nullptr, b = nullptr;
  float best = 1e30f;
  if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess && cudaGraphLaunch(g, st) == cudaSuccess) {
    for (int r = 0; r < 3; r++) {
      if (cudaEventRecord(a, st) != cudaSuccess || cudaGraphLaunch(g, st) != cudaSuccess ||
          cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess)
        break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      best = std::min(best, ms);
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return best;
}

// An autotuned plan carries the settings that were fastest for it alone on the GPU (autotune): for a
// plan with few modes that is often the partitioned z solve and small tiles, which buy latency with
// extra work.  In a batch graph the members share the GPU and throughput decides, so the first batch
// over a list of plans with autotuned members times its graph twice on scratch buffers of the
// members' sizes -- with every member's own settings, and with the shared-GPU settings for the
// autotuned ones (SettingsSwap) -- and returns which was faster (0 own, 1 shared).  It waits for
// earlier work on st, which may still use the members' workspaces, and allocates the scratch for
// the duration of the call; without the memory it keeps the members' own settings.
static int tune_batch(pp_plan* const* plans, int n, cudaStream_t st) {
  if (cudaStreamSynchronize(st) != cudaSuccess) return 0;
  std::vector<void*> fs(n, nullptr), us(n, nullptr);
  bool ok = true;
  for (int i = 0; i < n && ok; i++) {
    const bool f32 = (plans[i]->dtype == PP_MIXED_F32IO);
    const long long pts = (long long)plans[i]->nx * plans[i]->ny * plans[i]->nz;
    const size_t bytes = (size_t)pts * (f32 ? 4 : 8);
    ok = cudaMalloc(&fs[i], bytes) == cudaSuccess && cudaMalloc(&us[i], bytes) == cudaSuccess &&
         launch_fill(fs[i], pts, f32, st) == cudaSuccess;
  }
  int choice = 0;
  if (ok) {
    float t[2] = {1e30f, 1e30f};
    for (int v = 0; v < 2; v++) {
      SettingsSwap swap;
      if (v == 1) swap.apply(plans, n);
      cudaGraphExec_t g = nullptr;
      if (capture_batch(plans, fs.data(), us.data(), n, &g) == PP_OK) {
        t[v] = time_graph(g, st);
        cudaGraphExecDestroy(g);
      }
    }
    choice = (t[1] < t[0]) ? 1 : 0;
  }
  cudaStreamSynchronize(st);
  for (void* x : fs) if (x) cudaFree(x);
  for (void* x : us) if (x) cudaFree(x);
  (void)cudaGetLastError();  // a failed timing run leaves nothing for the caller's launches
  // the timing runs' status (scratch data) is not the caller's
  for (int i = 0; i < n; i++) cudaMemset(plans[i]->d_status, 0, sizeof(unsigned));
  return choice;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* pp_version(void) { return "pittpack-gb 0.1 (sm_103a)"; }

const char* pp_last_error_string(void) { return g_err.c_str(); }

pp_status pp_plan_create(pp_plan** out, int nx, int ny, int nz, const pp_bc bc[6], double dx, double dy, double dz,
                         pp_dtype dtype, const pp_plan_options* opt) {
  g_err.clear();
  if (!out) return fail(PP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!bc) return fail(PP_ERR_INVALID_ARG, "bc is NULL");
  if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
    return fail(PP_ERR_INVALID_ARG, "spacings must be positive and finite");
  if (dtype != PP_F64 && dtype != PP_MIXED_F64IO && dtype != PP_MIXED_F32IO)
    return fail(PP_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
  for (int i = 0; i < 6; i++)
    if (bc[i] != PP_BC_PERIODIC && bc[i] != PP_BC_NEUMANN && bc[i] != PP_BC_DIRICHLET)
      return fail(PP_ERR_INVALID_ARG, "bc[%d] = %d is not a boundary condition", i, (int)bc[i]);
  for (int a = 0; a < 3; a++)
    if ((bc[2 * a] == PP_BC_PERIODIC) != (bc[2 * a + 1] == PP_BC_PERIODIC))
      return fail(PP_ERR_BC_PAIRING, "axis %d: periodic must be given on both faces", a);
  if (opt) {
    if (opt->reserved[0]) return fail(PP_ERR_INVALID_ARG, "options.reserved must be zero");
    if (opt->z_method < 0 || opt->z_method > 2) return fail(PP_ERR_INVALID_ARG, "options.z_method must be 0, 1 or 2");
    const int zs = opt->z_split;
    if (zs != 0 && zs != 1 && zs != kZSplitRows[0] && zs != kZSplitRows[1] && zs != kZSplitRows[2])
      return fail(PP_ERR_INVALID_ARG, "options.z_split must be 0, 1, 8, 16 or 32 (got %d)", zs);
  }
  const int tmax = 512;
  if (opt) {
    for (int v : {opt->threads_x, opt->threads_y, opt->threads_x_inv, opt->threads_y_inv})
      if (v < 0 || (v && (v % 32 || v > tmax)))
        return fail(PP_ERR_INVALID_ARG, "options: thread counts must be multiples of 32, at most %d", tmax);
    for (int v : {opt->lines_x, opt->cols_y, opt->lines_x_inv, opt->cols_y_inv})
      if (v < 0) return fail(PP_ERR_INVALID_ARG, "options: lines / columns per CTA must be >= 0");
  }
  for (int v : {nx, ny})
    if (v < 2 || v > 4096 || v % 2 || !smooth2357(v))
      return fail(PP_ERR_UNSUPPORTED_SIZE, "nx, ny must be even 2^a 3^b 5^c 7^d in [2, 4096] (got %d x %d)", nx, ny);
  bool zper = (bc[4] == PP_BC_PERIODIC);
  if (nz < (zper ? 3 : 2) || nz > (1 << 20))
    return fail(PP_ERR_UNSUPPORTED_SIZE, "nz = %d out of range (>= 2, periodic z >= 3)", nz);
  if ((long long)nx * ny > (1LL << 30) || (long long)nx * ny * nz > (1LL << 36))
    return fail(PP_ERR_UNSUPPORTED_SIZE, "grid too large");
  // line counts of one launch are 32-bit: x lines ny*nz, y lines (nx + 2)*nz at most
  if ((long long)ny * nz >= (1LL << 31) || (long long)(nx + 2) * nz >= (1LL << 31))
    return fail(PP_ERR_UNSUPPORTED_SIZE, "too many lines per launch (ny*nz and (nx+2)*nz must be < 2^31)");

  // periodic z by transform: nz must be a length the line kernels transform (7-smooth, <= 4096)
  const bool zfft_ok = zper && nz <= 4096 && smooth2357(nz);
  const int zreq = opt ? opt->z_method : 0;
  if (zreq == 2 && !zfft_ok)
    return fail(PP_ERR_UNSUPPORTED_SIZE, "z_method 2 (transform) needs periodic z and nz = 2^a 3^b 5^c 7^d <= 4096");
  // partitioned z solve (non-periodic z; ignored for periodic z): at most 512 chunks per line
  const int sreq = (opt && !zper) ? opt->z_split : 0;
  if (sreq > 1) {
    int G, lgG, P;
    if (!zpart_shape(nz, sreq, &G, &lgG, &P))
      return fail(PP_ERR_UNSUPPORTED_SIZE, "z_split %d: nz = %d needs more than 512 chunks per line", sreq, nz);
  }

  pp_plan* p = new (std::nothrow) pp_plan();
  if (!p) return fail(PP_ERR_OUT_OF_MEMORY, "host allocation failed");
  memset(p, 0, sizeof *p);
  p->nx = nx; p->ny = ny; p->nz = nz;
  for (int i = 0; i < 6; i++) p->bc[i] = bc[i];
  p->dx = dx; p->dy = dy; p->dz = dz;
  p->dtype = dtype;
  p->kx = axis_kind(bc[0], bc[1]);
  p->ky = axis_kind(bc[2], bc[3]);
  p->layout = (p->kx == AX_P) ? 0 : (p->ky == AX_P ? 1 : 2);
  p->singular = true;
  for (int i = 0; i < 6; i++)
    if (bc[i] == PP_BC_DIRICHLET) p->singular = false;
  p->elem = (dtype == PP_F64) ? 8 : 4;
  // x-spectral rows are padded to a multiple of 4 reals so every row starts 16-byte aligned
  p->xrow = (((p->kx == AX_P) ? (long long)nx + 2 : nx) + 3) / 4 * 4;
  p->xplane = p->xrow * ny;
  if (p->layout == 1) p->splane = 2LL * nx * (ny / 2 + 1);
  else p->splane = p->xplane;
  p->zscale = dz * dz * axis_weight(p->kx, nx) * axis_weight(p->ky, ny);

  pp_status s;
  if ((s = axis_tables(p, p->kx, nx, false, p->fx, &p->d_tw_x, &p->d_aux_x)) != PP_OK) { free_plan(p); return s; }
  if ((s = axis_tables(p, p->ky, ny, p->layout == 0, p->fy, &p->d_tw_y, &p->d_aux_y)) != PP_OK) { free_plan(p); return s; }
  if ((s = z_tables(p)) != PP_OK) { free_plan(p); return s; }
  p->zfft_ok = zfft_ok;
  if (p->zfft_ok && (s = zfft_tables(p)) != PP_OK) { free_plan(p); return s; }
  p->zmethod = (zreq == 2) ? ZM_FFT : ZM_SM;
  p->zsplit = (sreq > 1) ? sreq : 1;
  choose_shapes(p, opt);

  p->buf_bytes = (size_t)std::max(p->xplane, p->splane) * nz * p->elem;
  cudaError_t e = cudaMalloc(&p->bufA, p->buf_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&p->bufB, p->buf_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_status, 4 * sizeof(unsigned));
  if (e != cudaSuccess) {
    free_plan(p);
    return fail(PP_ERR_OUT_OF_MEMORY, "workspace allocation of 2 x %zu bytes failed: %s", p->buf_bytes,
                cudaGetErrorString(e));
  }
  cudaMemset(p->d_status, 0, 4 * sizeof(unsigned));
  if (opt && opt->autotune) {
    pp_status ts = autotune(p, zreq == 0, sreq == 0 && !zper);
    if (ts != PP_OK) { free_plan(p); return ts; }
    p->tuned = true;
    p->z_tuned = zper ? (zreq == 0 && zfft_ok) : (sreq == 0);
  }
  *out = p;
  return PP_OK;
}

pp_status pp_plan_destroy(pp_plan* plan) {
  if (!plan) return PP_OK;
  cudaDeviceSynchronize();
  evict_plan(plan);
  free_plan(plan);
  return PP_OK;
}

pp_status pp_solve(pp_plan* p, const void* f, void* u, pp_stream_t stream) {
  if (!p || !f || !u) return fail(PP_ERR_INVALID_ARG, "NULL plan or pointer");
  return run_pipeline(p, f, u, 0, (cudaStream_t)stream);
}

pp_status pp_solve_adjoint(pp_plan* p, const void* g, void* gf, pp_stream_t stream) {
  if (!p || !g || !gf) return fail(PP_ERR_INVALID_ARG, "NULL plan or pointer");
  // S = X^-1 Y^-1 T^-1 W Y X with W the constant inverse weight; S^T = X^T Y^T W T^-T Y^-T X^-T.
  // The unnormalised syntheses are the transposes of the analyses up to the per-mode
  // multiplicities that the weight absorbs, so the transposed pipeline runs the same line
  // kernels around the transposed tridiagonal factorisation.
  return run_pipeline(p, g, gf, 1, (cudaStream_t)stream);
}

pp_status pp_fold_bc(pp_plan* p, const void* f_in, void* f_out, const void* const g[6], pp_stream_t stream) {
  if (!p || !f_in || !f_out || !g) return fail(PP_ERR_INVALID_ARG, "NULL plan or pointer");
  for (int face = 0; face < 6; face++)
    if (g[face] && p->bc[face] == PP_BC_PERIODIC)
      return fail(PP_ERR_INVALID_ARG, "face %d is periodic and takes no data", face);
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = (p->dtype == PP_MIXED_F32IO);
  if (f_in != f_out) {
    const size_t bytes = (size_t)p->nx * p->ny * p->nz * (f32 ? 4 : 8);
    cudaError_t e = cudaMemcpyAsync(f_out, f_in, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(PP_ERR_CUDA, "copy of the source: %s", cudaGetErrorString(e));
  }
  const double h[3] = {p->dx, p->dy, p->dz};
  for (int face = 0; face < 6; face++) {
    if (!g[face]) continue;
    const double hn = h[face >> 1];
    // L_g(0) next to the face: ghost / h^2 with ghost 2 g (Dirichlet) or h q (Neumann)
    const double coef = (p->bc[face] == PP_BC_DIRICHLET) ? 2.0 * (1.0 / (hn * hn)) : hn * (1.0 / (hn * hn));
    cudaError_t e = launch_fold_face(f_out, g[face], p->nx, p->ny, p->nz, face, coef, f32, st);
    if (e != cudaSuccess) return fail(PP_ERR_CUDA, "face %d launch: %s", face, cudaGetErrorString(e));
  }
  return PP_OK;
}

pp_status pp_solve_refined(pp_plan* p, const void* f, void* u, pp_stream_t stream) {
  if (!p || !f || !u) return fail(PP_ERR_INVALID_ARG, "NULL plan or pointer");
  if (p->dtype != PP_MIXED_F64IO) return fail(PP_ERR_INVALID_ARG, "refinement needs a PP_MIXED_F64IO plan");
  if (f == u) return fail(PP_ERR_INVALID_ARG, "u must not alias f for the refined solve");
  if (!p->d_resid) {
    size_t bytes = 2 * (size_t)p->nx * p->ny * p->nz * sizeof(float);
    cudaError_t e = cudaMalloc(&p->d_resid, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_mean, (kMeanParts + 1) * sizeof(float2));
    if (e != cudaSuccess) return fail(PP_ERR_OUT_OF_MEMORY, "residual buffer (%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  return solve_refined_core(p, f, u, p->d_resid, p->d_mean, (float2*)p->d_mean + kMeanParts, (cudaStream_t)stream);
}

pp_status pp_solve_batched(pp_plan* const* plans, const void* const* f, void* const* u, int n, pp_stream_t stream) {
  if (n < 0 || (n > 0 && (!plans || !f || !u))) return fail(PP_ERR_INVALID_ARG, "bad batch arguments");
  if (n == 0) return PP_OK;
  for (int i = 0; i < n; i++)
    if (!plans[i] || !f[i] || !u[i]) return fail(PP_ERR_INVALID_ARG, "batch member %d: NULL plan or pointer", i);
  std::vector<const void*> key;
  key.reserve(3 * (size_t)n);
  for (int i = 0; i < n; i++) key.push_back(plans[i]);
  for (int i = 0; i < n; i++) key.push_back(f[i]);
  for (int i = 0; i < n; i++) key.push_back(u[i]);
  cudaStream_t st = (cudaStream_t)stream;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batch_cache.size(); i++) {
      if (g_batch_cache[i].key == key) {
        BatchGraph hit = g_batch_cache[i];
        g_batch_cache.erase(g_batch_cache.begin() + i);
        g_batch_cache.push_back(hit);
        CUDA_OK(cudaGraphLaunch(hit.exec, st));
        return PP_OK;
      }
    }
  }
  // Launch settings of the batch: tuned once per list of plans that includes autotuned members.
  int choice = 0;
  bool any_tuned = false;
  for (int i = 0; i < n; i++) any_tuned |= plans[i]->tuned;
  // No tuning while the caller's stream is being captured: it waits for the stream and launches
  // timing runs, neither of which belongs in the caller's graph (the members keep their settings,
  // and a later call outside a capture tunes the list).
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  if (any_tuned && (cudaStreamIsCapturing(st, &cap_status) != cudaSuccess || cap_status != cudaStreamCaptureStatusNone))
    any_tuned = false;
  if (any_tuned) {
    const std::vector<const pp_plan*> pk(plans, plans + n);
    bool found = false;
    {
      std::lock_guard<std::mutex> lk(g_batch_mu);
      for (const BatchChoice& c : g_batch_choice)
        if (c.plans == pk) { choice = c.choice; found = true; break; }
    }
    if (!found) {
      choice = tune_batch(plans, n, st);
      std::lock_guard<std::mutex> lk(g_batch_mu);
      if (g_batch_choice.size() >= kBatchChoiceMax) g_batch_choice.erase(g_batch_choice.begin());
      g_batch_choice.push_back(BatchChoice{pk, choice});
    }
  }
  cudaGraphExec_t exec = nullptr;
  pp_status s;
  {
    SettingsSwap swap;
    if (choice == 1) swap.apply(plans, n);
    s = capture_batch(plans, f, u, n, &exec);
  }
  if (s != PP_OK) return s;
  cudaError_t e = cudaGraphLaunch(exec, st);
  if (e != cudaSuccess) {
    cudaGraphExecDestroy(exec);
    return fail(PP_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (g_batch_cache.size() >= kBatchCacheMax) {
    // the evicted graph may still be running on some stream: destroy it only after it finished
    cudaStreamSynchronize(st);
    cudaGraphExecDestroy(g_batch_cache.front().exec);
    g_batch_cache.erase(g_batch_cache.begin());
  }
  g_batch_cache.push_back(BatchGraph{std::move(key), exec});
  return PP_OK;
}

pp_status pp_solve_host(pp_plan* p, const void* f_host, void* u_host, pp_stream_t stream) {
  if (!p || !f_host || !u_host) return fail(PP_ERR_INVALID_ARG, "NULL plan or pointer");
  const size_t elem = (p->dtype == PP_MIXED_F32IO ? 4 : 8);
  const size_t plane = (size_t)p->nx * p->ny * elem;
  const size_t bytes = plane * p->nz;
  if (!p->d_host_f) {
    cudaError_t e = cudaMalloc(&p->d_host_f, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_host_u, bytes);
    if (e != cudaSuccess) return fail(PP_ERR_OUT_OF_MEMORY, "staging buffers: %s", cudaGetErrorString(e));
  }
  if (!p->host_cs[0]) {
    for (cudaStream_t& s : p->host_cs) CUDA_OK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    for (cudaEvent_t& e : p->host_ev) CUDA_OK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  // Plane chunks: the host->device copy of chunk c (copy engines, two streams) overlaps the x/y
  // forward transforms of the chunks before it; after the z solve, the device->host copy of
  // chunk c overlaps the inverse transforms of the chunks after it.
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t* ev = p->host_ev;
  const int C = std::min(kHostChunks, p->nz);
  auto z0 = [&](int c) { return (int)((long long)c * p->nz / C); };
  char* df = static_cast<char*>(p->d_host_f);
  char* du = static_cast<char*>(p->d_host_u);
  CUDA_OK(cudaEventRecord(ev[2 * kHostChunks], st));  // earlier work on st (users of the staging buffers)
  for (cudaStream_t s : p->host_cs) CUDA_OK(cudaStreamWaitEvent(s, ev[2 * kHostChunks], 0));
  for (int c = 0; c < C; c++) {
    const size_t off = (size_t)z0(c) * plane, n = (size_t)(z0(c + 1) - z0(c)) * plane;
    CUDA_OK(cudaMemcpyAsync(df + off, static_cast<const char*>(f_host) + off, n, cudaMemcpyHostToDevice, p->host_cs[c % 2]));
    CUDA_OK(cudaEventRecord(ev[c], p->host_cs[c % 2]));
  }
  for (int c = 0; c < C; c++) {
    CUDA_OK(cudaStreamWaitEvent(st, ev[c], 0));
    for (int stage : {0, 1}) {
      pp_status s = run_stage(p, stage, df, du, 0, st, z0(c), z0(c + 1) - z0(c));
      if (s != PP_OK) return s;
    }
  }
  pp_status s = run_stage(p, 2, df, du, 0, st);
  if (s != PP_OK) return s;
  for (int c = 0; c < C; c++) {
    for (int stage : {3, 4}) {
      s = run_stage(p, stage, df, du, 0, st, z0(c), z0(c + 1) - z0(c));
      if (s != PP_OK) return s;
    }
    CUDA_OK(cudaEventRecord(ev[kHostChunks + c], st));
    CUDA_OK(cudaStreamWaitEvent(p->host_cs[c % 2], ev[kHostChunks + c], 0));
    const size_t off = (size_t)z0(c) * plane, n = (size_t)(z0(c + 1) - z0(c)) * plane;
    CUDA_OK(cudaMemcpyAsync(static_cast<char*>(u_host) + off, du + off, n, cudaMemcpyDeviceToHost, p->host_cs[c % 2]));
  }
  for (int k = 0; k < 2; k++) {
    CUDA_OK(cudaEventRecord(ev[2 * kHostChunks + 1 + k], p->host_cs[k]));
    CUDA_OK(cudaStreamWaitEvent(st, ev[2 * kHostChunks + 1 + k], 0));
  }
  CUDA_OK(cudaStreamSynchronize(st));
  (void)bytes;
  return PP_OK;
}

pp_status pp_run_stage(pp_plan* p, int stage, const void* f, void* u, pp_stream_t stream) {
  if (!p) return fail(PP_ERR_INVALID_ARG, "NULL plan");
  if ((stage == 0 && !f) || (stage == 4 && !u)) return fail(PP_ERR_INVALID_ARG, "NULL pointer for stage %d", stage);
  return run_stage(p, stage, f, u, 0, (cudaStream_t)stream);
}

pp_status pp_plan_status(pp_plan* p) {
  if (!p) return fail(PP_ERR_INVALID_ARG, "NULL plan");
  unsigned v = 0;
  CUDA_OK(cudaMemcpy(&v, p->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  CUDA_OK(cudaMemset(p->d_status, 0, sizeof(unsigned)));
  if (v & kStatusRange)
    return fail(PP_ERR_RANGE,
                "a solve met values outside the range of full accuracy: largest scaled z input below 2^-100, "
                "largest z output above 2^124/(nx ny) = %.3g, or non-finite values; scale f by a power of two",
                0x1p124 / ((double)p->nx * (double)p->ny));
  if (v) return fail(PP_ERR_INTERNAL, "device reported status bits 0x%x", v);
  return PP_OK;
}

pp_status pp_plan_launch_shapes(const pp_plan* p, int out[8]) {
  if (!p || !out) return fail(PP_ERR_INVALID_ARG, "NULL plan or pointer");
  const int v[8] = {p->threads_x[0], p->lpc_x[0], p->threads_y[0], p->lpc_y[0],
                    p->threads_y[1], p->lpc_y[1], p->threads_x[1], p->lpc_x[1]};
  for (int i = 0; i < 8; i++) out[i] = v[i];
  return PP_OK;
}

pp_status pp_plan_z_method(const pp_plan* p, int* out) {
  if (!p || !out) return fail(PP_ERR_INVALID_ARG, "NULL plan or pointer");
  *out = (p->bc[4] != PP_BC_PERIODIC) ? 0 : (p->zmethod == ZM_FFT ? 2 : 1);
  return PP_OK;
}

pp_status pp_plan_z_split(const pp_plan* p, int* out) {
  if (!p || !out) return fail(PP_ERR_INVALID_ARG, "NULL plan or pointer");
  *out = (p->bc[4] == PP_BC_PERIODIC) ? 1 : p->zsplit;
  return PP_OK;
}

size_t pp_plan_device_bytes(const pp_plan* p) {
  if (!p) return 0;
  return 2 * p->buf_bytes;
}

}  // extern "C"
