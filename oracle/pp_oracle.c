/*
 * pp_oracle.c -- CPU oracle for the FFT / tridiagonal Poisson solve of
 * Hasbestan & Senocak, "PittPack: An Open-Source Poisson's Equation Solver
 * for Extreme-Scale Computing with Accelerators" (arXiv 1909.05423).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never calls it.  It shares no code, tables or helpers with
 * the CUDA library.
 *
 * Everything is FP64 and naive: every line transform is the O(N^2) sum that
 * defines it, every tridiagonal system is solved by the textbook Thomas
 * algorithm.  The steps follow the paper's method section in order:
 *
 *   1. forward transform along x, then along y, the transform chosen per
 *      boundary condition (Sec. "Boundary Conditions": periodic -> DFT,
 *      Neumann -> DCT-II ("DCT10"), Dirichlet -> DST-II ("DST10"); table of
 *      forward/backward transforms);  mixed Dirichlet/Neumann faces on one
 *      axis use the type-IV sine/cosine transform (the paper only notes that
 *      eight DCT/DST variants exist; the type-IV pair is the one whose basis
 *      satisfies a Dirichlet face at one end and a Neumann face at the other);
 *   2. for every (kx,ky) pair a tridiagonal system along z whose diagonal is
 *      shifted by the sum of the per-axis eigenvalues (Table "Eigenvalues"),
 *      solved with the Thomas algorithm (Sec. "Thomas Algorithm"), periodic z
 *      by the Sherman-Morrison modification, the singular mode of an
 *      all-Neumann/periodic problem by removing the source mean
 *      (Sec. "Well-posedness");
 *   3. inverse transforms along y, then x.
 *
 * Discretisation (Sec. "Mathematical Formulation"): cell-centred 7-point
 * Laplacian, sum over axes (u[i+1]-2u[i]+u[i-1])/h^2 = f, ghost cells by the
 * face condition: periodic wraps, Neumann copies the interior value
 * (u[-1]=u[0]), homogeneous Dirichlet extrapolates linearly to a zero face
 * value (u[-1]=-u[0]).
 *
 * Layout: real arrays [nz][ny][nx], x fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_BC_P = 0, OR_BC_N = 1, OR_BC_D = 2 };
/* axis kinds: both faces periodic, Neumann-Neumann, Dirichlet-Dirichlet,
 * Dirichlet(low)-Neumann(high), Neumann(low)-Dirichlet(high) */
enum { AX_P = 0, AX_NN = 1, AX_DD = 2, AX_DN = 3, AX_ND = 4 };

int oracle_axis_kind(int lo, int hi) {
  if (lo == OR_BC_P || hi == OR_BC_P) return (lo == OR_BC_P && hi == OR_BC_P) ? AX_P : -1;
  if (lo == OR_BC_N && hi == OR_BC_N) return AX_NN;
  if (lo == OR_BC_D && hi == OR_BC_D) return AX_DD;
  if (lo == OR_BC_D && hi == OR_BC_N) return AX_DN;
  if (lo == OR_BC_N && hi == OR_BC_D) return AX_ND;
  return -1;
}

/* Forward basis b_k(n) of one axis: Y_k = sum_n u_n b_k(n).
 *  P : exp(-2 pi i n k / N)                       (Sec. "Periodic Boundary Condition")
 *  NN: cos(pi (n+1/2) k / N)                       (DCT10 definition)
 *  DD: sin(pi (n+1/2)(k+1) / N)                    (DST10 definition)
 *  DN: sin(pi (n+1/2)(k+1/2) / N)   type IV, odd at the low face, even at the high face
 *  ND: cos(pi (n+1/2)(k+1/2) / N)   type IV, even at the low face, odd at the high face
 * Angles are reduced exactly in integers before calling cos/sin. */
static void basis(int kind, int N, int k, int n, double* re, double* im) {
  const double PI = 3.14159265358979323846;
  long long m;
  double th;
  switch (kind) {
    case AX_P:
      m = ((long long)n * k) % N;
      th = 2.0 * PI * (double)m / (double)N;
      *re = cos(th); *im = -sin(th); return;
    case AX_NN:
      m = ((long long)(2 * n + 1) * k) % (4LL * N);
      th = PI * (double)m / (2.0 * N);
      *re = cos(th); *im = 0.0; return;
    case AX_DD:
      m = ((long long)(2 * n + 1) * (k + 1)) % (4LL * N);
      th = PI * (double)m / (2.0 * N);
      *re = sin(th); *im = 0.0; return;
    case AX_DN:
      m = ((long long)(2 * n + 1) * (2 * k + 1)) % (8LL * N);
      th = PI * (double)m / (4.0 * N);
      *re = sin(th); *im = 0.0; return;
    default: /* AX_ND */
      m = ((long long)(2 * n + 1) * (2 * k + 1)) % (8LL * N);
      th = PI * (double)m / (4.0 * N);
      *re = cos(th); *im = 0.0; return;
  }
}

/* Inverse weight c_k = 1 / ||b_k||^2, so that u_n = sum_k c_k Y_k conj(b_k(n)). */
static double inv_weight(int kind, int N, int k) {
  switch (kind) {
    case AX_P: return 1.0 / N;
    case AX_NN: return (k == 0) ? 1.0 / N : 2.0 / N;
    case AX_DD: return (k == N - 1) ? 1.0 / N : 2.0 / N;
    default: return 2.0 / N;
  }
}

/* Per-axis eigenvalue of the 1-D second difference (unit spacing), Table "Eigenvalues";
 * the mixed D/N axis follows from the type-IV basis: -2 + 2 cos(pi (k+1/2) / N). */
double oracle_eigenvalue(int kind, int N, int k) {
  const double PI = 3.14159265358979323846;
  switch (kind) {
    case AX_P: return -2.0 + 2.0 * cos(2.0 * PI * (double)k / N);
    case AX_NN: return -2.0 + 2.0 * cos(PI * (double)k / N);
    case AX_DD: return -2.0 + 2.0 * cos(PI * (double)(k + 1) / N);
    default: return -2.0 + 2.0 * cos(PI * (2.0 * k + 1.0) / (2.0 * N));
  }
}

/* Dense basis table, N x N complex, row k. */
static void make_table(int kind, int N, double* tre, double* tim) {
  for (int k = 0; k < N; k++)
    for (int n = 0; n < N; n++) basis(kind, N, k, n, &tre[(size_t)k * N + n], &tim[(size_t)k * N + n]);
}

/* One line, forward: out_k = sum_n in_n b_k(n) (complex in, complex out). */
static void line_fwd(int N, const double* tre, const double* tim, const double* ire, const double* iim,
                     size_t stride, double* ore, double* oim) {
  for (int k = 0; k < N; k++) {
    double sr = 0.0, si = 0.0;
    const double* br = tre + (size_t)k * N;
    const double* bi = tim + (size_t)k * N;
    for (int n = 0; n < N; n++) {
      double xr = ire[n * stride], xi = iim[n * stride];
      sr += xr * br[n] - xi * bi[n];
      si += xr * bi[n] + xi * br[n];
    }
    ore[k] = sr; oim[k] = si;
  }
}

/* One line, inverse: out_n = sum_k c_k in_k conj(b_k(n)). */
static void line_inv(int kind, int N, const double* tre, const double* tim, const double* ire, const double* iim,
                     size_t stride, double* ore, double* oim) {
  for (int n = 0; n < N; n++) {
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < N; k++) {
      double c = inv_weight(kind, N, k);
      double br = tre[(size_t)k * N + n], bi = -tim[(size_t)k * N + n];
      double xr = ire[k * stride], xi = iim[k * stride];
      sr += c * (xr * br - xi * bi);
      si += c * (xr * bi + xi * br);
    }
    ore[n] = sr; oim[n] = si;
  }
}

/* Public single-line transforms (used by the transform pins). */
int oracle_line_forward(int kind, int N, const double* ire, const double* iim, double* ore, double* oim) {
  if (kind < 0 || kind > 4 || N < 1) return -1;
  double* t = (double*)malloc(sizeof(double) * 2 * (size_t)N * N);
  if (!t) return -2;
  make_table(kind, N, t, t + (size_t)N * N);
  line_fwd(N, t, t + (size_t)N * N, ire, iim, 1, ore, oim);
  free(t);
  return 0;
}
int oracle_line_inverse(int kind, int N, const double* ire, const double* iim, double* ore, double* oim) {
  if (kind < 0 || kind > 4 || N < 1) return -1;
  double* t = (double*)malloc(sizeof(double) * 2 * (size_t)N * N);
  if (!t) return -2;
  make_table(kind, N, t, t + (size_t)N * N);
  line_inv(kind, N, t, t + (size_t)N * N, ire, iim, 1, ore, oim);
  free(t);
  return 0;
}

/* Textbook Thomas algorithm (Sec. "Thomas Algorithm"): a = sub-diagonal (a[0] unused),
 * b = diagonal, c = super-diagonal (c[n-1] unused).  Forward elimination with the
 * multipliers cp[i] = c[i] / (b[i] - a[i] cp[i-1]), then back substitution
 * x[i] = dp[i] - cp[i] x[i+1].  No pivoting.  Work arrays of length n. */
int oracle_thomas(int n, const double* a, const double* b, const double* c, const double* d, double* x) {
  if (n < 1) return -1;
  double* cp = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  if (!cp) return -2;
  double* dp = cp + n;
  cp[0] = (n > 1) ? c[0] / b[0] : 0.0;
  dp[0] = d[0] / b[0];
  for (int i = 1; i < n; i++) {
    double m = b[i] - a[i] * cp[i - 1];
    cp[i] = (i < n - 1) ? c[i] / m : 0.0;
    dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; i--) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  return 0;
}

/* Cyclic tridiagonal system (periodic z) by the Sherman-Morrison modification named in
 * Sec. "Thomas Algorithm": A = A' + u v^T with corner entries alpha = A[n-1][0] and
 * beta = A[0][n-1], u = (gamma,0..0,alpha), v = (1,0..0,beta/gamma), gamma = -b[0];
 * A' is A with b'[0] = b[0]-gamma, b'[n-1] = b[n-1]-alpha*beta/gamma and no corners.
 * Then x = y - (v.y)/(1+v.z) z with A'y = d, A'z = u.  Requires n >= 2. */
int oracle_cyclic(int n, const double* a, const double* b, const double* c, double alpha, double beta,
                  const double* d, double* x) {
  if (n < 2) return -1;
  double* w = (double*)malloc(sizeof(double) * 4 * (size_t)n);
  if (!w) return -2;
  double* bb = w; double* uu = w + n; double* y = w + 2 * n; double* z = w + 3 * n;
  double gamma = -b[0];
  memcpy(bb, b, sizeof(double) * n);
  bb[0] = b[0] - gamma;
  bb[n - 1] = b[n - 1] - alpha * beta / gamma;
  for (int i = 0; i < n; i++) uu[i] = 0.0;
  uu[0] = gamma; uu[n - 1] = alpha;
  oracle_thomas(n, a, bb, c, d, y);
  oracle_thomas(n, a, bb, c, uu, z);
  double fac = (y[0] + beta * y[n - 1] / gamma) / (1.0 + z[0] + beta * z[n - 1] / gamma);
  for (int i = 0; i < n; i++) x[i] = y[i] - fac * z[i];
  free(w);
  return 0;
}

/* Solve one z-line for one (kx,ky) pair: sum of the per-axis eigenvalues lam (already
 * divided by h^2) on the diagonal, 1/dz^2 off the diagonal, end rows from the z faces.
 * singular != 0: the lam = 0 mode with no Dirichlet face anywhere (Sec. "Well-posedness"):
 * the source mean is removed, row 0 is dropped and u[0] pinned to 0, the rest solved,
 * and the result shifted to zero mean. */
static void zline(int nz, int zlo, int zhi, double dz, double lam, int singular, const double* d,
                  double* x, double* work) {
  double* a = work; double* b = work + nz; double* c = work + 2 * nz; double* dd = work + 3 * nz;
  double h2 = 1.0 / (dz * dz);
  for (int k = 0; k < nz; k++) { a[k] = h2; c[k] = h2; b[k] = -2.0 * h2 + lam; dd[k] = d[k]; }
  int periodic = (zlo == OR_BC_P);
  if (!periodic) {
    b[0] += (zlo == OR_BC_N) ? h2 : -h2;
    b[nz - 1] += (zhi == OR_BC_N) ? h2 : -h2;
  }
  if (singular) {
    double mean = 0.0;
    for (int k = 0; k < nz; k++) mean += dd[k];
    mean /= nz;
    for (int k = 0; k < nz; k++) dd[k] -= mean;
    x[0] = 0.0;
    if (nz > 1) {
      /* rows 1..nz-1 with u[0] = 0 known; for periodic z row nz-1 also touches u[0] = 0 */
      oracle_thomas(nz - 1, a + 1, b + 1, c + 1, dd + 1, x + 1);
    }
    double m = 0.0;
    for (int k = 0; k < nz; k++) m += x[k];
    m /= nz;
    for (int k = 0; k < nz; k++) x[k] -= m;
    return;
  }
  if (periodic) oracle_cyclic(nz, a, b, c, h2, h2, dd, x);
  else oracle_thomas(nz, a, b, c, dd, x);
}

/* Cell-centred 7-point Laplacian A_h u with the ghost rules above (Sec. "Mathematical Formulation"). */
static inline double ghost(int bc, double inside) { return (bc == OR_BC_N) ? inside : -inside; }

static inline double lap_at(int nx, int ny, int nz, const int* bc, double ix2, double iy2, double iz2,
                            const double* u, int i, int j, int k) {
  size_t sy = (size_t)nx, sz = (size_t)nx * ny;
  size_t p = (size_t)k * sz + (size_t)j * sy + i;
  double c = u[p], xm, xp, ym, yp, zm, zp;
  if (i > 0) xm = u[p - 1]; else xm = (bc[0] == OR_BC_P) ? u[p + nx - 1] : ghost(bc[0], c);
  if (i < nx - 1) xp = u[p + 1]; else xp = (bc[1] == OR_BC_P) ? u[p - (nx - 1)] : ghost(bc[1], c);
  if (j > 0) ym = u[p - sy]; else ym = (bc[2] == OR_BC_P) ? u[p + (ny - 1) * sy] : ghost(bc[2], c);
  if (j < ny - 1) yp = u[p + sy]; else yp = (bc[3] == OR_BC_P) ? u[p - (ny - 1) * sy] : ghost(bc[3], c);
  if (k > 0) zm = u[p - sz]; else zm = (bc[4] == OR_BC_P) ? u[p + (nz - 1) * sz] : ghost(bc[4], c);
  if (k < nz - 1) zp = u[p + sz]; else zp = (bc[5] == OR_BC_P) ? u[p - (nz - 1) * sz] : ghost(bc[5], c);
  return (xm - 2.0 * c + xp) * ix2 + (ym - 2.0 * c + yp) * iy2 + (zm - 2.0 * c + zp) * iz2;
}

static int check_bc(const int* bc) {
  for (int a = 0; a < 3; a++)
    if (oracle_axis_kind(bc[2 * a], bc[2 * a + 1]) < 0) return -3;
  return 0;
}

int oracle_laplacian(int nx, int ny, int nz, const int* bc, double dx, double dy, double dz, const double* u,
                     double* out) {
  if (nx < 1 || ny < 1 || nz < 1) return -1;
  if (check_bc(bc)) return -3;
  double ix2 = 1.0 / (dx * dx), iy2 = 1.0 / (dy * dy), iz2 = 1.0 / (dz * dz);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++)
        out[(size_t)k * nx * ny + (size_t)j * nx + i] = lap_at(nx, ny, nz, bc, ix2, iy2, iz2, u, i, j, k);
  return 0;
}

/* A_h u at a list of flat cell indices (for sampled checks on large grids). */
int oracle_laplacian_at(int nx, int ny, int nz, const int* bc, double dx, double dy, double dz, const double* u,
                        const int64_t* idx, int64_t count, double* out) {
  if (check_bc(bc)) return -3;
  double ix2 = 1.0 / (dx * dx), iy2 = 1.0 / (dy * dy), iz2 = 1.0 / (dz * dz);
  int64_t total = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < count; q++) {
    int64_t p = idx[q];
    if (p < 0 || p >= total) { out[q] = NAN; continue; }
    int i = (int)(p % nx), j = (int)((p / nx) % ny), k = (int)(p / ((int64_t)nx * ny));
    out[q] = lap_at(nx, ny, nz, bc, ix2, iy2, iz2, u, i, j, k);
  }
  return 0;
}

/* Faces with data (the step before the path in an incompressible-flow projection; the paper's
 * Sec. "Boundary Conditions" defines the Dirichlet ghost by linear extrapolation to the face
 * value): Dirichlet face value g gives the ghost u_ghost = 2 g - u_inside; Neumann data q is the
 * outward normal derivative, (u_ghost - u_inside) / h = q, so u_ghost = u_inside + h q.  With these
 * ghosts the stencil is an affine operator L_g u = A_h u + L_g(0).
 * g[face]: NULL (homogeneous face) or the face's values, faces x-,x+,y-,y+,z-,z+; x faces are
 * [nz][ny], y faces [nz][nx], z faces [ny][nx].  A periodic face must have no data. */
static double face_value(const double* const* g, int face, int i, int j, int k, int nx, int ny) {
  const double* v = g ? g[face] : NULL;
  if (!v) return 0.0;
  if (face < 2) return v[(size_t)k * ny + j];
  if (face < 4) return v[(size_t)k * nx + i];
  return v[(size_t)j * nx + i];
}

static inline double ghost_g(int bc, double inside, double data, double h) {
  return (bc == OR_BC_N) ? inside + h * data : 2.0 * data - inside;
}

/* L_g u: the 7-point Laplacian with the data ghosts above. */
int oracle_laplacian_g(int nx, int ny, int nz, const int* bc, double dx, double dy, double dz,
                       const double* const* g, const double* u, double* out) {
  if (nx < 1 || ny < 1 || nz < 1) return -1;
  if (check_bc(bc)) return -3;
  for (int f = 0; f < 6; f++)
    if (g && g[f] && bc[f] == OR_BC_P) return -4;
  double ix2 = 1.0 / (dx * dx), iy2 = 1.0 / (dy * dy), iz2 = 1.0 / (dz * dz);
  size_t sy = (size_t)nx, sz = (size_t)nx * ny;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        size_t p = (size_t)k * sz + (size_t)j * sy + i;
        double c = u[p], xm, xp, ym, yp, zm, zp;
        if (i > 0) xm = u[p - 1];
        else xm = (bc[0] == OR_BC_P) ? u[p + nx - 1] : ghost_g(bc[0], c, face_value(g, 0, i, j, k, nx, ny), dx);
        if (i < nx - 1) xp = u[p + 1];
        else xp = (bc[1] == OR_BC_P) ? u[p - (nx - 1)] : ghost_g(bc[1], c, face_value(g, 1, i, j, k, nx, ny), dx);
        if (j > 0) ym = u[p - sy];
        else ym = (bc[2] == OR_BC_P) ? u[p + (ny - 1) * sy] : ghost_g(bc[2], c, face_value(g, 2, i, j, k, nx, ny), dy);
        if (j < ny - 1) yp = u[p + sy];
        else yp = (bc[3] == OR_BC_P) ? u[p - (ny - 1) * sy] : ghost_g(bc[3], c, face_value(g, 3, i, j, k, nx, ny), dy);
        if (k > 0) zm = u[p - sz];
        else zm = (bc[4] == OR_BC_P) ? u[p + (nz - 1) * sz] : ghost_g(bc[4], c, face_value(g, 4, i, j, k, nx, ny), dz);
        if (k < nz - 1) zp = u[p + sz];
        else zp = (bc[5] == OR_BC_P) ? u[p - (nz - 1) * sz] : ghost_g(bc[5], c, face_value(g, 5, i, j, k, nx, ny), dz);
        out[p] = (xm - 2.0 * c + xp) * ix2 + (ym - 2.0 * c + yp) * iy2 + (zm - 2.0 * c + zp) * iz2;
      }
  return 0;
}

/* The problem L_g u = f is A_h u = f - L_g(0): out = f - L_g(0) (out may alias f). */
int oracle_fold_bc(int nx, int ny, int nz, const int* bc, double dx, double dy, double dz,
                   const double* const* g, const double* f, double* out) {
  size_t n = (size_t)nx * ny * nz;
  double* zero = (double*)calloc(n, sizeof(double));
  double* l0 = (double*)malloc(n * sizeof(double));
  if (!zero || !l0) { free(zero); free(l0); return -2; }
  int rc = oracle_laplacian_g(nx, ny, nz, bc, dx, dy, dz, g, zero, l0);
  if (rc == 0)
    for (size_t p = 0; p < n; p++) out[p] = f[p] - l0[p];
  free(zero);
  free(l0);
  return rc;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* The full solve (steps 1-3 above).  f and u are real [nz][ny][nx]; u may alias f.
 * Returns 0, or a negative code for bad arguments / allocation failure. */
int oracle_solve(int nx, int ny, int nz, const int* bc, double dx, double dy, double dz, const double* f,
                 double* u) {
  if (nx < 1 || ny < 1 || nz < 2) return -1;
  if (check_bc(bc)) return -3;
  int kx = oracle_axis_kind(bc[0], bc[1]), ky = oracle_axis_kind(bc[2], bc[3]);
  int zlo = bc[4], zhi = bc[5];
  if (oracle_axis_kind(zlo, zhi) < 0) return -3;
  size_t nxy = (size_t)nx * ny, n = nxy * nz;
  double* re = (double*)malloc(sizeof(double) * n);
  double* im = (double*)calloc(n, sizeof(double));
  double* tx = (double*)malloc(sizeof(double) * 2 * (size_t)nx * nx);
  double* ty = (double*)malloc(sizeof(double) * 2 * (size_t)ny * ny);
  if (!re || !im || !tx || !ty) { free(re); free(im); free(tx); free(ty); return -2; }
  memcpy(re, f, sizeof(double) * n);
  make_table(kx, nx, tx, tx + (size_t)nx * nx);
  make_table(ky, ny, ty, ty + (size_t)ny * ny);
  int singular = (bc[0] != OR_BC_D && bc[1] != OR_BC_D && bc[2] != OR_BC_D && bc[3] != OR_BC_D &&
                  bc[4] != OR_BC_D && bc[5] != OR_BC_D);
  int err = 0;

  /* 1a. forward x on every (j,k) line */
#pragma omp parallel
  {
    double* buf = (double*)malloc(sizeof(double) * 2 * (size_t)(nx > ny ? nx : ny));
    if (!buf) {
#pragma omp atomic write
      err = 1;
    } else {
#pragma omp for collapse(2) schedule(static)
      for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++) {
          size_t o = (size_t)k * nxy + (size_t)j * nx;
          line_fwd(nx, tx, tx + (size_t)nx * nx, re + o, im + o, 1, buf, buf + nx);
          memcpy(re + o, buf, sizeof(double) * nx);
          memcpy(im + o, buf + nx, sizeof(double) * nx);
        }
      /* 1b. forward y on every (kx,k) line */
#pragma omp for collapse(2) schedule(static)
      for (int k = 0; k < nz; k++)
        for (int i = 0; i < nx; i++) {
          size_t o = (size_t)k * nxy + i;
          line_fwd(ny, ty, ty + (size_t)ny * ny, re + o, im + o, (size_t)nx, buf, buf + ny);
          for (int j = 0; j < ny; j++) { re[o + (size_t)j * nx] = buf[j]; im[o + (size_t)j * nx] = buf[ny + j]; }
        }
      free(buf);
    }
  }
  if (err) { free(re); free(im); free(tx); free(ty); return -2; }

  /* 2. tridiagonal solve along z for every (kx,ky) */
#pragma omp parallel
  {
    double* work = (double*)malloc(sizeof(double) * 8 * (size_t)nz);
    if (!work) {
#pragma omp atomic write
      err = 1;
    } else {
      double* dr = work + 4 * nz; double* xr = work + 5 * nz; double* di = work + 6 * nz; double* xi = work + 7 * nz;
#pragma omp for collapse(2) schedule(static)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          double lam = oracle_eigenvalue(kx, nx, i) / (dx * dx) + oracle_eigenvalue(ky, ny, j) / (dy * dy);
          int sing = singular && i == 0 && j == 0;
          size_t o = (size_t)j * nx + i;
          for (int k = 0; k < nz; k++) { dr[k] = re[o + (size_t)k * nxy]; di[k] = im[o + (size_t)k * nxy]; }
          zline(nz, zlo, zhi, dz, lam, sing, dr, xr, work);
          zline(nz, zlo, zhi, dz, lam, sing, di, xi, work);
          for (int k = 0; k < nz; k++) { re[o + (size_t)k * nxy] = xr[k]; im[o + (size_t)k * nxy] = xi[k]; }
        }
      free(work);
    }
  }
  if (err) { free(re); free(im); free(tx); free(ty); return -2; }

  /* 3. inverse y, then inverse x */
#pragma omp parallel
  {
    double* buf = (double*)malloc(sizeof(double) * 2 * (size_t)(nx > ny ? nx : ny));
    if (!buf) {
#pragma omp atomic write
      err = 1;
    } else {
#pragma omp for collapse(2) schedule(static)
      for (int k = 0; k < nz; k++)
        for (int i = 0; i < nx; i++) {
          size_t o = (size_t)k * nxy + i;
          line_inv(ky, ny, ty, ty + (size_t)ny * ny, re + o, im + o, (size_t)nx, buf, buf + ny);
          for (int j = 0; j < ny; j++) { re[o + (size_t)j * nx] = buf[j]; im[o + (size_t)j * nx] = buf[ny + j]; }
        }
#pragma omp for collapse(2) schedule(static)
      for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++) {
          size_t o = (size_t)k * nxy + (size_t)j * nx;
          line_inv(kx, nx, tx, tx + (size_t)nx * nx, re + o, im + o, 1, buf, buf + nx);
          memcpy(re + o, buf, sizeof(double) * nx);
          memcpy(im + o, buf + nx, sizeof(double) * nx);
        }
      free(buf);
    }
  }
  if (!err) memcpy(u, re, sizeof(double) * n);
  free(re); free(im); free(tx); free(ty);
  return err ? -2 : 0;
}
