/* Matrix-free FP64 boundary-integral mobility in plain C (test infrastructure).
 *
 * Same discrete operator as oracle/bie.py, for sizes where the dense matrix
 * does not fit: straight double loops over all node pairs (OpenMP over
 * targets), restarted GMRES with modified Gram-Schmidt and Givens rotations.
 * Only the tests and the CPU-baseline leg of the bench use it; the GPU
 * library shares nothing with it.
 *
 * Operator (Sec. 2, Fig. 1 of the paper; stand-in described in oracle/bie.py):
 *   (K phi)_p = sum_{q != p} w_q T(x_p - x_q, n_q)(phi_q - phi_p),
 *   T(r, n) v = -(3 / 4 pi) r (r.n)(r.v) / |r|^5,
 *   (P phi) = weighted orthogonal projection onto each body's rigid modes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double PI = 3.14159265358979323846;

/* Solve the 6x6 system G c = m in place by Gaussian elimination with partial pivoting. */
static void solve6(double G[6][6], double m[6]) {
  for (int k = 0; k < 6; k++) {
    int piv = k;
    for (int i = k + 1; i < 6; i++) if (fabs(G[i][k]) > fabs(G[piv][k])) piv = i;
    if (piv != k) {
      for (int j = 0; j < 6; j++) { double t = G[k][j]; G[k][j] = G[piv][j]; G[piv][j] = t; }
      double t = m[k]; m[k] = m[piv]; m[piv] = t;
    }
    for (int i = k + 1; i < 6; i++) {
      double f = G[i][k] / G[k][k];
      for (int j = k; j < 6; j++) G[i][j] -= f * G[k][j];
      m[i] -= f * m[k];
    }
  }
  for (int k = 5; k >= 0; k--) {
    double s = m[k];
    for (int j = k + 1; j < 6; j++) s -= G[k][j] * m[j];
    m[k] = s / G[k][k];
  }
}

/* Rigid basis vector k (0..5) at relative position xi: e_k or e_{k-3} x xi. */
static void rigid_mode(int k, const double* xi, double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  if (k < 3) { out[k] = 1.0; return; }
  double e[3] = {0, 0, 0};
  e[k - 3] = 1.0;
  out[0] = e[1] * xi[2] - e[2] * xi[1];
  out[1] = e[2] * xi[0] - e[0] * xi[2];
  out[2] = e[0] * xi[1] - e[1] * xi[0];
}

/* Rigid coefficients c (6 per body) of P phi: c = G^{-1} Psi^T W phi. */
void mf_rigid_coeffs(int M, int ns, const double* x, const double* w, const double* centers,
                     const double* phi, double* coeff) {
  for (int i = 0; i < M; i++) {
    double G[6][6] = {{0}}, m[6] = {0};
    for (int q = i * ns; q < (i + 1) * ns; q++) {
      double xi[3] = {x[3 * q] - centers[3 * i], x[3 * q + 1] - centers[3 * i + 1],
                      x[3 * q + 2] - centers[3 * i + 2]};
      double psi[6][3];
      for (int k = 0; k < 6; k++) rigid_mode(k, xi, psi[k]);
      for (int k = 0; k < 6; k++) {
        m[k] += w[q] * (psi[k][0] * phi[3 * q] + psi[k][1] * phi[3 * q + 1] + psi[k][2] * phi[3 * q + 2]);
        for (int l = 0; l < 6; l++)
          G[k][l] += w[q] * (psi[k][0] * psi[l][0] + psi[k][1] * psi[l][1] + psi[k][2] * psi[l][2]);
      }
    }
    solve6(G, m);
    for (int k = 0; k < 6; k++) coeff[6 * i + k] = m[k];
  }
}

/* out = (K + P) phi for N = M * ns nodes; with Cself (3 ns x 3 ns, row-major, or
 * NULL) also out_b += Cself phi_b on every body b (the accurate self-interaction). */
void mf_apply(int M, int ns, const double* x, const double* nrm, const double* w,
              const double* centers, const double* Cself, const double* phi, double* out) {
  int N = M * ns;
  const double c = -3.0 / (4.0 * PI);
#pragma omp parallel for schedule(dynamic, 16)
  for (int p = 0; p < N; p++) {
    double acc[3] = {0, 0, 0};
    for (int q = 0; q < N; q++) {
      if (q == p) continue;
      double r[3] = {x[3 * p] - x[3 * q], x[3 * p + 1] - x[3 * q + 1], x[3 * p + 2] - x[3 * q + 2]};
      double d[3] = {phi[3 * q] - phi[3 * p], phi[3 * q + 1] - phi[3 * p + 1],
                     phi[3 * q + 2] - phi[3 * p + 2]};
      double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      double rn = r[0] * nrm[3 * q] + r[1] * nrm[3 * q + 1] + r[2] * nrm[3 * q + 2];
      double rd = r[0] * d[0] + r[1] * d[1] + r[2] * d[2];
      double s = c * w[q] * rn * rd / (r2 * r2 * sqrt(r2));
      acc[0] += s * r[0];
      acc[1] += s * r[1];
      acc[2] += s * r[2];
    }
    out[3 * p] = acc[0];
    out[3 * p + 1] = acc[1];
    out[3 * p + 2] = acc[2];
  }
  double* coeff = (double*)malloc(sizeof(double) * 6 * M);
  mf_rigid_coeffs(M, ns, x, w, centers, phi, coeff);
  for (int p = 0; p < N; p++) {
    int i = p / ns;
    double xi[3] = {x[3 * p] - centers[3 * i], x[3 * p + 1] - centers[3 * i + 1],
                    x[3 * p + 2] - centers[3 * i + 2]};
    for (int k = 0; k < 6; k++) {
      double psi[3];
      rigid_mode(k, xi, psi);
      for (int a = 0; a < 3; a++) out[3 * p + a] += coeff[6 * i + k] * psi[a];
    }
  }
  free(coeff);
  if (Cself) {
    int nb = 3 * ns;
#pragma omp parallel for
    for (int i = 0; i < M; i++)
      for (int r = 0; r < nb; r++) {
        double s = 0.0;
        for (int c2 = 0; c2 < nb; c2++) s += Cself[(size_t)r * nb + c2] * phi[(size_t)i * nb + c2];
        out[(size_t)i * nb + r] += s;
      }
  }
}

/* rhs = -S[F, T] at the nodes (Stokeslet and rotlet of every body). */
void mf_stokeslet_rhs(int M, int ns, const double* x, const double* centers, const double* FT,
                      double mu, double* rhs) {
  int N = M * ns;
#pragma omp parallel for
  for (int p = 0; p < N; p++) {
    double u[3] = {0, 0, 0};
    for (int j = 0; j < M; j++) {
      double r[3] = {x[3 * p] - centers[3 * j], x[3 * p + 1] - centers[3 * j + 1],
                     x[3 * p + 2] - centers[3 * j + 2]};
      double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
      const double* F = FT + 6 * j;
      const double* T = FT + 6 * j + 3;
      double rF = r[0] * F[0] + r[1] * F[1] + r[2] * F[2];
      double TxR[3] = {T[1] * r[2] - T[2] * r[1], T[2] * r[0] - T[0] * r[2], T[0] * r[1] - T[1] * r[0]};
      for (int a = 0; a < 3; a++)
        u[a] += (F[a] / rr + r[a] * rF / (rr * rr * rr)) / (8 * PI * mu) + TxR[a] / (8 * PI * mu * rr * rr * rr);
    }
    for (int a = 0; a < 3; a++) rhs[3 * p + a] = -u[a];
  }
}

/* Restarted GMRES(m) with MGS for (K + P) phi = rhs, phi starting at 0.
 * Stops when ||rhs - (K+P) phi|| <= tol ||rhs||; returns the iteration count
 * (negative if maxit was reached). */
int mf_gmres(int M, int ns, const double* x, const double* nrm, const double* w,
             const double* centers, const double* Cself, const double* rhs, double* phi, double tol, int m,
             int maxit) {
  int n = 3 * M * ns;
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (m + 1));
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * m);
  double* sn = (double*)malloc(sizeof(double) * m);
  double* g = (double*)malloc(sizeof(double) * (m + 1));
  double* y = (double*)malloc(sizeof(double) * m);
  double* wv = (double*)malloc(sizeof(double) * n);
  double bnorm = 0;
  for (int i = 0; i < n; i++) bnorm += rhs[i] * rhs[i];
  bnorm = sqrt(bnorm);
  memset(phi, 0, sizeof(double) * n);
  int total = 0;
  if (bnorm == 0.0) goto done;
  for (;;) {
    mf_apply(M, ns, x, nrm, w, centers, Cself, phi, wv);
    double beta = 0;
    for (int i = 0; i < n; i++) { wv[i] = rhs[i] - wv[i]; beta += wv[i] * wv[i]; }
    beta = sqrt(beta);
    if (beta <= tol * bnorm) goto done;
    for (int i = 0; i < n; i++) V[i] = wv[i] / beta;
    memset(g, 0, sizeof(double) * (m + 1));
    g[0] = beta;
    int j;
    for (j = 0; j < m; j++) {
      mf_apply(M, ns, x, nrm, w, centers, Cself, V + (size_t)j * n, wv);
      total++;
      for (int k = 0; k <= j; k++) {
        double h = 0;
        for (int i = 0; i < n; i++) h += wv[i] * V[(size_t)k * n + i];
        H[k * m + j] = h;
        for (int i = 0; i < n; i++) wv[i] -= h * V[(size_t)k * n + i];
      }
      double hn = 0;
      for (int i = 0; i < n; i++) hn += wv[i] * wv[i];
      hn = sqrt(hn);
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < n; i++) V[(size_t)(j + 1) * n + i] = wv[i] / hn;
      for (int k = 0; k < j; k++) {
        double a = H[k * m + j], b = H[(k + 1) * m + j];
        H[k * m + j] = cs[k] * a + sn[k] * b;
        H[(k + 1) * m + j] = -sn[k] * a + cs[k] * b;
      }
      double a = H[j * m + j], b = H[(j + 1) * m + j];
      double rr = sqrt(a * a + b * b);
      cs[j] = a / rr;
      sn[j] = b / rr;
      H[j * m + j] = rr;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (fabs(g[j + 1]) <= tol * bnorm || total >= maxit) { j++; break; }
    }
    for (int k = j - 1; k >= 0; k--) {
      double s = g[k];
      for (int l = k + 1; l < j; l++) s -= H[k * m + l] * y[l];
      y[k] = s / H[k * m + k];
    }
    for (int k = 0; k < j; k++)
      for (int i = 0; i < n; i++) phi[i] += y[k] * V[(size_t)k * n + i];
    if (total >= maxit) { total = -total; break; }
  }
done:
  free(V); free(H); free(cs); free(sn); free(g); free(y); free(wv);
  return total;
}
