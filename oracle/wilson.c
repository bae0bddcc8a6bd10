/*
 * Plain FP64 CPU oracle of the Wilson-Dirac operator and of the pseudofermion force.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library (paper_1010_5636_gb300) may call,
 * link or include this file; only tests/, the smoke check and the CPU-baseline leg of
 * bench.py use it, through oracle/wilson.py.
 *
 * Everything here is written for a reader checking it against the paper by eye:
 * scalar loops over lexicographic sites, full 4x4 gamma matrices (no half-spinor
 * trick), explicit 3x3 complex matrix-vector products, C99 complex arithmetic.
 *
 * Operator (Sec. 2.1, definition of D_W and Q):
 *   D_W phi(x) = (4+m) phi(x) - 1/2 sum_{mu=+-0..+-3} U_mu(x) (1 - gamma_mu) phi(x+mu)
 *   Q = gamma5 D_W,  U_{-mu}(x) = U_mu(x-mu)^{-1} = U_mu(x-mu)^dagger,  gamma_{-mu} = -gamma_mu.
 *
 * Layouts (canonical, interleaved re/im doubles):
 *   lattice extents dims = {T, L1, L2, L3}; x = (x0,x1,x2,x3), mu = 0 is time;
 *   lex(x) = x3 + L3*(x2 + L2*(x1 + L1*x0));
 *   spinor  psi[lex][spin 4][colour 3]          (V*12 complex)
 *   links   U[mu][lex][row 3][col 3]            (4*V*9 complex)
 *   force   F[mu][lex][a = 1..8]                (4*V*8 doubles, coefficient of T^a = lambda^a/2)
 * Boundary conditions: periodic, optionally antiperiodic in time (a hop across the
 * t boundary picks up a factor -1).
 */
#include <complex.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Gamma matrices in the chiral basis, gamma5 = gamma0 gamma1 gamma2 gamma3 = diag(1,1,-1,-1).
 * In 2x2 blocks: gamma0 = [[0,-1],[-1,0]], gamma_k = [[0,-i sigma_k],[i sigma_k,0]].
 * Index 4 holds gamma5.  Written out entry by entry; tests check the Clifford algebra,
 * hermiticity and the product formula for gamma5 numerically. */
static cplx G[5][4][4];
static int G_ready = 0;

static void init_gammas(void) {
  if (G_ready) return;
  memset(G, 0, sizeof(G));
  /* gamma0 */
  G[0][0][2] = -1; G[0][1][3] = -1; G[0][2][0] = -1; G[0][3][1] = -1;
  /* gamma1: -i sigma1 = [[0,-i],[-i,0]] upper right, i sigma1 lower left */
  G[1][0][3] = -I; G[1][1][2] = -I; G[1][2][1] = I; G[1][3][0] = I;
  /* gamma2: -i sigma2 = [[0,-1],[1,0]] upper right, i sigma2 = [[0,1],[-1,0]] lower left */
  G[2][0][3] = -1; G[2][1][2] = 1; G[2][2][1] = 1; G[2][3][0] = -1;
  /* gamma3: -i sigma3 = [[-i,0],[0,i]] upper right, i sigma3 = [[i,0],[0,-i]] lower left */
  G[3][0][2] = -I; G[3][1][3] = I; G[3][2][0] = I; G[3][3][1] = -I;
  /* gamma5 */
  G[4][0][0] = 1; G[4][1][1] = 1; G[4][2][2] = -1; G[4][3][3] = -1;
  G_ready = 1;
}

void oracle_gamma(int mu, double* out /* [4][4][2] */) {
  init_gammas();
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      out[2 * (4 * a + b)] = creal(G[mu][a][b]);
      out[2 * (4 * a + b) + 1] = cimag(G[mu][a][b]);
    }
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static void coords(const int* d, long lex, int x[4]) {
  x[3] = (int)(lex % d[3]); lex /= d[3];
  x[2] = (int)(lex % d[2]); lex /= d[2];
  x[1] = (int)(lex % d[1]); lex /= d[1];
  x[0] = (int)lex;
}

static long lexof(const int* d, const int x[4]) {
  return x[3] + (long)d[3] * (x[2] + (long)d[2] * (x[1] + (long)d[1] * x[0]));
}

/* lex index of x + dir*mu (dir = +1 or -1) with periodic wrap; *sign gets the boundary factor. */
static long hop_site(const int* d, int antiperiodic_t, const int x[4], int mu, int dir, double* sign) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[mu] += dir;
  *sign = 1.0;
  if (y[mu] < 0) { y[mu] += d[mu]; if (mu == 0 && antiperiodic_t) *sign = -1.0; }
  if (y[mu] >= d[mu]) { y[mu] -= d[mu]; if (mu == 0 && antiperiodic_t) *sign = -1.0; }
  return lexof(d, y);
}

#define LINK(U, V, mu, s) ((const cplx*)(U) + ((size_t)(mu) * (V) + (size_t)(s)) * 9)
#define SPIN(p, s) ((const cplx*)(p) + (size_t)(s) * 12)

/* D_W (gamma5 = 0) or Q = gamma5 D_W (gamma5 = 1), Sec. 2.1. */
static void apply_wilson(const int* dims, int antiperiodic_t, double m, const double* U, const double* in,
                         double* out, int with_gamma5) {
  init_gammas();
  const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s) {
    int x[4];
    coords(dims, s, x);
    cplx acc[4][3];
    memset(acc, 0, sizeof(acc));
    for (int mu = 0; mu < 4; ++mu) {
      /* forward: U_mu(x) (1 - gamma_mu) psi(x + mu) */
      double sf;
      long xf = hop_site(dims, antiperiodic_t, x, mu, +1, &sf);
      const cplx* pf = SPIN(in, xf);
      const cplx* Uf = LINK(U, V, mu, s);
      cplx t[4][3];
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
          cplx v = 0;
          for (int b = 0; b < 4; ++b) v += ((a == b ? 1.0 : 0.0) - G[mu][a][b]) * pf[3 * b + i];
          t[a][i] = sf * v;
        }
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) acc[a][i] += Uf[3 * i + j] * t[a][j];
      /* backward: U_{-mu}(x) (1 - gamma_{-mu}) psi(x - mu) = U_mu(x-mu)^dagger (1 + gamma_mu) psi(x - mu) */
      double sb;
      long xb = hop_site(dims, antiperiodic_t, x, mu, -1, &sb);
      const cplx* pb = SPIN(in, xb);
      const cplx* Ub = LINK(U, V, mu, xb);
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
          cplx v = 0;
          for (int b = 0; b < 4; ++b) v += ((a == b ? 1.0 : 0.0) + G[mu][a][b]) * pb[3 * b + i];
          t[a][i] = sb * v;
        }
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) acc[a][i] += conj(Ub[3 * j + i]) * t[a][j];
    }
    const cplx* p0 = SPIN(in, s);
    cplx dw[4][3];
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) dw[a][i] = (4.0 + m) * p0[3 * a + i] - 0.5 * acc[a][i];
    cplx* o = (cplx*)out + (size_t)s * 12;
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        if (!with_gamma5) { o[3 * a + i] = dw[a][i]; continue; }
        cplx v = 0;
        for (int b = 0; b < 4; ++b) v += G[4][a][b] * dw[b][i];
        o[3 * a + i] = v;
      }
  }
}

void oracle_apply_Q(const int* dims, int antiperiodic_t, double m, const double* U, const double* in, double* out) {
  apply_wilson(dims, antiperiodic_t, m, U, in, out, 1);
}

void oracle_apply_DW(const int* dims, int antiperiodic_t, double m, const double* U, const double* in,
                     double* out) {
  apply_wilson(dims, antiperiodic_t, m, U, in, out, 0);
}

/* Gell-Mann matrices lambda^a, a = 1..8 (stored at index a-1). */
static cplx LAM[8][3][3];
static int LAM_ready = 0;
static void init_gellmann(void) {
  if (LAM_ready) return;
  memset(LAM, 0, sizeof(LAM));
  LAM[0][0][1] = 1; LAM[0][1][0] = 1;
  LAM[1][0][1] = -I; LAM[1][1][0] = I;
  LAM[2][0][0] = 1; LAM[2][1][1] = -1;
  LAM[3][0][2] = 1; LAM[3][2][0] = 1;
  LAM[4][0][2] = -I; LAM[4][2][0] = I;
  LAM[5][1][2] = 1; LAM[5][2][1] = 1;
  LAM[6][1][2] = -I; LAM[6][2][1] = I;
  const double r3 = 0.57735026918962576451; /* 1/sqrt(3) */
  LAM[7][0][0] = r3; LAM[7][1][1] = r3; LAM[7][2][2] = -2.0 * r3;
  LAM_ready = 1;
}

void oracle_gellmann(int a /* 1..8 */, double* out /* [3][3][2] */) {
  init_gellmann();
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      out[2 * (3 * i + j)] = creal(LAM[a - 1][i][j]);
      out[2 * (3 * i + j) + 1] = cimag(LAM[a - 1][i][j]);
    }
}

/*
 * Force of S = phi^dagger (Q^2)^{-1} phi with respect to the links, given X = (Q^2)^{-1} phi
 * and Y = Q X.  Under U_mu(x) -> exp(i w T^a) U_mu(x) with T^a = lambda^a / 2,
 *   dS/dw = -2 Re(Y^dagger dQ X) = -Im tr[T^a (A1 - A2)],
 *   A1 = U_mu(x) sum_alpha [(1 - gamma_mu) X(x+mu)]_alpha [gamma5 Y(x)]_alpha^dagger,
 *   A2 = sum_alpha [(1 + gamma_mu) X(x)]_alpha [U_mu(x) gamma5 Y(x+mu)]_alpha^dagger,
 * where [.]_alpha is the colour 3-vector of spin component alpha and the sum runs over alpha.
 * (Derivation: dQ = -1/2 gamma5 dH from the definition of D_W; dU = i w T U, dU^dagger = -i w U^dagger T.)
 */
void oracle_force(const int* dims, int antiperiodic_t, const double* U, const double* Xd, const double* Yd,
                  double* F) {
  init_gammas();
  init_gellmann();
  const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s) {
    int x[4];
    coords(dims, s, x);
    for (int mu = 0; mu < 4; ++mu) {
      double sf;
      long xf = hop_site(dims, antiperiodic_t, x, mu, +1, &sf);
      const cplx* Um = LINK(U, V, mu, s);
      const cplx* Xx = SPIN(Xd, s);
      const cplx* Xf = SPIN(Xd, xf);
      const cplx* Yx = SPIN(Yd, s);
      const cplx* Yf = SPIN(Yd, xf);
      cplx pX[4][3], mX[4][3], g5Yx[4][3], g5Yf[4][3], UgYf[4][3];
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
          cplx v1 = 0, v2 = 0, v3 = 0, v4 = 0;
          for (int b = 0; b < 4; ++b) {
            v1 += ((a == b ? 1.0 : 0.0) - G[mu][a][b]) * Xf[3 * b + i];
            v2 += ((a == b ? 1.0 : 0.0) + G[mu][a][b]) * Xx[3 * b + i];
            v3 += G[4][a][b] * Yx[3 * b + i];
            v4 += G[4][a][b] * Yf[3 * b + i];
          }
          mX[a][i] = sf * v1; /* (1 - gamma_mu) X(x+mu) with boundary factor */
          pX[a][i] = v2;      /* (1 + gamma_mu) X(x) */
          g5Yx[a][i] = v3;
          g5Yf[a][i] = sf * v4;
        }
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
          cplx v = 0;
          for (int j = 0; j < 3; ++j) v += Um[3 * i + j] * g5Yf[a][j];
          UgYf[a][i] = v;
        }
      /* B = sum_alpha mX_alpha g5Yx_alpha^dagger;  A1 = U B;  A2 = sum_alpha pX_alpha UgYf_alpha^dagger */
      cplx B[3][3], A1[3][3], A2[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          cplx b = 0, a2 = 0;
          for (int a = 0; a < 4; ++a) {
            b += mX[a][i] * conj(g5Yx[a][j]);
            a2 += pX[a][i] * conj(UgYf[a][j]);
          }
          B[i][j] = b;
          A2[i][j] = a2;
        }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          cplx v = 0;
          for (int k = 0; k < 3; ++k) v += Um[3 * i + k] * B[k][j];
          A1[i][j] = v;
        }
      double* f = F + ((size_t)mu * V + (size_t)s) * 8;
      for (int c = 0; c < 8; ++c) {
        cplx tr = 0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) tr += 0.5 * LAM[c][i][j] * (A1[j][i] - A2[j][i]);
        f[c] = -cimag(tr);
      }
    }
  }
}
