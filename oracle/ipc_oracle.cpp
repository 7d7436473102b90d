// Plain FP64 CPU oracle for one IPC time step (Eq. 3, §III-C.2).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file; only the tests, the smoke check and the CPU-baseline leg of
// the benchmark use it.  It shares no code with the CUDA library.
//
// Everything is written as the plain definition: no blocking, no fusion, no
// spatial acceleration.  Candidate pairs are found by brute force over all
// (surface vertex, surface triangle) and (surface edge, surface edge) pairs.
// The two brute-force pair loops are spread over OpenMP threads in chunks of
// the outer index; each chunk's pairs are kept apart and concatenated in chunk
// order afterwards, so the output (pairs, their order, the minimum time of
// impact) is the same as the serial loop's for any thread count
// (orc_set_threads).
// Compiled with -ffp-contract=off so every product and sum rounds exactly as
// written.
//
// Conventions
//   * 3x3 matrices are row-major: M[3*i + j] = M_ij.
//   * vec(F) is column-major: vec[3*j + i] = F_ij (columns f_0, f_1, f_2).
//   * A stencil of 4 points is stored vertex-major, x[3*k + d].
//   * 12x12 (and 9x9) matrices are row-major.
//
// Readings of points the paper leaves open (it names the models only):
//   * Elasticity (§III-C.1, "Stable Neo-Hookean"): the rest-stable form
//       Psi = mu/2 (tr F^T F - 3) - mu (J - 1) + lam/2 (J - 1)^2,
//     which is zero with zero stress at F = I and at any rotation; callers pass
//     lam = (first Lame parameter) + mu so the small-strain limit has the
//     given Young modulus and Poisson ratio.
//   * Barrier (Eq. 3, "log-barrier"): on squared distance s,
//       b(s) = -(s - sh)^2 ln(s / sh) for 0 < s < sh, 0 otherwise, sh = dhat^2,
//     scaled by kappa; edge-edge pairs carry the IPC mollifier on
//     c = |e_a x e_b|^2 with eps_x = 1e-3 |ea_rest|^2 |eb_rest|^2.
//   * Friction (Eq. 3, "smoothly mollified friction"): lagged IPC friction,
//     D = mu lambda f0(|P u|), f0 the C1 cubic below eps = eps_v dt.
//   * Continuous collision detection (§III-C.1): additive CCD with a
//     minimum-separation fraction s (0.1), conservative advancement.
//   * PSD projection: cyclic Jacobi eigen-decomposition, negative eigenvalues
//     clamped to zero.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <vector>
#include <omp.h>

extern "C" {

// Threads of the brute-force pair loops (<= 0: OpenMP's default).
static int g_threads = 0;
void orc_set_threads(int n) { g_threads = n; }
int orc_get_threads(void) { return g_threads > 0 ? g_threads : omp_get_max_threads(); }

// ---------------------------------------------------------------------------
// small dense helpers
// ---------------------------------------------------------------------------

static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void sub3(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
// [w]x, the matrix with [w]x v = w x v
static inline void skew(const double* w, double* M) {
  M[0] = 0;     M[1] = -w[2]; M[2] = w[1];
  M[3] = w[2];  M[4] = 0;     M[5] = -w[0];
  M[6] = -w[1]; M[7] = w[0];  M[8] = 0;
}
static inline void matmul3(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (n <= 12).
// On return A is (numerically) diagonal, V holds the eigenvectors as columns.
// Sweeps stop when the off-diagonal Frobenius norm is below 1e-15 of the
// whole matrix norm, or after 50 sweeps.
int orc_jacobi_eigen(int n, double* A, double* V) {
  for (int i = 0; i < n * n; ++i) V[i] = 0;
  for (int i = 0; i < n; ++i) V[i * n + i] = 1;
  double total = 0;
  for (int i = 0; i < n * n; ++i) total += A[i] * A[i];
  if (total == 0) return 0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += 2 * A[p * n + q] * A[p * n + q];
    if (off <= 1e-30 * total) return sweep;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
        double c = 1 / std::sqrt(t * t + 1);
        double s = t * c;
        // A <- J^T A J with J the rotation in the (p, q) plane
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  return 50;
}

// H <- V max(Lambda, 0) V^T, the nearest PSD matrix in Frobenius norm.
void orc_project_psd(int n, double* H) {
  double A[144], V[144];
  std::memcpy(A, H, sizeof(double) * n * n);
  orc_jacobi_eigen(n, A, V);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0;
      for (int k = 0; k < n; ++k) {
        double lk = A[k * n + k];
        if (lk > 0) s += V[i * n + k] * lk * V[j * n + k];
      }
      H[i * n + j] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double m = 0.5 * (H[i * n + j] + H[j * n + i]);
      H[i * n + j] = m;
      H[j * n + i] = m;
    }
}

// ---------------------------------------------------------------------------
// Stable Neo-Hookean (reading above), per deformation gradient
// ---------------------------------------------------------------------------

// psi, P = dPsi/dF (row-major 3x3), H = d2Psi/dvec(F)^2 (9x9, column-major vec).
void orc_snh(const double* F, double mu, double lam, int project, double* psi, double* P, double* H) {
  double f[3][3];  // f[j] = column j of F
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) f[j][i] = F[3 * i + j];
  double c[3][3];  // cofactor columns: dJ/df_j
  cross3(f[1], f[2], c[0]);
  cross3(f[2], f[0], c[1]);
  cross3(f[0], f[1], c[2]);
  double J = dot3(f[0], c[0]);
  double Ic = 0;
  for (int i = 0; i < 9; ++i) Ic += F[i] * F[i];
  *psi = 0.5 * mu * (Ic - 3.0) - mu * (J - 1.0) + 0.5 * lam * (J - 1.0) * (J - 1.0);
  double kJ = lam * (J - 1.0) - mu;  // coefficient of dJ/dF in P and of d2J/dF2 in H
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P[3 * i + j] = mu * F[3 * i + j] + kJ * c[j][i];
  if (!H) return;
  double g[9];
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) g[3 * j + i] = c[j][i];
  for (int a = 0; a < 9; ++a)
    for (int b = 0; b < 9; ++b) H[9 * a + b] = (a == b ? mu : 0.0) + lam * g[a] * g[b];
  // d2J/(df_a df_b): block (0,1) = -[f2]x, (0,2) = [f1]x, (1,2) = -[f0]x, symmetric.
  double S[9];
  const int blocks[3][3] = {{0, 1, 2}, {0, 2, 1}, {1, 2, 0}};
  const double sign[3] = {-1.0, 1.0, -1.0};
  for (int k = 0; k < 3; ++k) {
    int a = blocks[k][0], b = blocks[k][1], w = blocks[k][2];
    skew(f[w], S);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double v = kJ * sign[k] * S[3 * i + j];
        H[9 * (3 * a + i) + (3 * b + j)] += v;
        H[9 * (3 * b + j) + (3 * a + i)] += v;
      }
  }
  if (project) orc_project_psd(9, H);
}

// One tet: energy V*Psi, gradient and 12x12 Hessian w.r.t. its 4 vertices.
// B = Dm^{-1} (row-major), Dm = [X1 - X0, X2 - X0, X3 - X0].
void orc_tet(const double* x, const double* B, double vol, double mu, double lam, int project, double* E,
             double* g, double* H) {
  double Ds[9];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) Ds[3 * i + k] = x[3 * (k + 1) + i] - x[i];
  double F[9];
  matmul3(Ds, B, F);
  double psi, P[9], H9[81];
  orc_snh(F, mu, lam, project, &psi, P, H ? H9 : nullptr);
  *E = vol * psi;
  // dF[:,j]/dx_a = C[a][j] I with C[k+1][j] = B[k][j], C[0][j] = -sum_k B[k][j]
  double C[4][3];
  for (int j = 0; j < 3; ++j) {
    C[0][j] = 0;
    for (int k = 0; k < 3; ++k) {
      C[k + 1][j] = B[3 * k + j];
      C[0][j] -= B[3 * k + j];
    }
  }
  for (int a = 0; a < 4; ++a)
    for (int i = 0; i < 3; ++i) {
      double s = 0;
      for (int j = 0; j < 3; ++j) s += C[a][j] * P[3 * i + j];
      g[3 * a + i] = vol * s;
    }
  if (!H) return;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
          double s = 0;
          for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l) s += C[a][j] * C[b][l] * H9[9 * (3 * j + i) + (3 * l + k)];
          H[12 * (3 * a + i) + (3 * b + k)] = vol * s;
        }
}

// All tets.  E (scalar) and g (3 nv) are accumulated.  Hv receives nt x 144
// values (tet-major, row-major 12x12); the caller maps them to DOF indices.
void orc_elastic_all(int nt, const int* tets, const double* Bs, const double* vols, const double* mus,
                     const double* lams, const double* x, int project, double* E, double* g, double* Hv) {
  double xs[12], ge[12], He[144], Ee;
  for (int e = 0; e < nt; ++e) {
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) xs[3 * a + d] = x[3 * tets[4 * e + a] + d];
    orc_tet(xs, Bs + 9 * e, vols[e], mus[e], lams[e], project, &Ee, ge, Hv ? He : nullptr);
    *E += Ee;
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) g[3 * tets[4 * e + a] + d] += ge[3 * a + d];
    if (Hv) std::memcpy(Hv + 144 * (size_t)e, He, sizeof(He));
  }
}

// ---------------------------------------------------------------------------
// squared distances with derivatives (stencil of 4 points, 12 DOFs)
// ---------------------------------------------------------------------------

// Adds coefficient-mapped derivatives of a function of "difference" variables
// u_m = sum_a cm[a] x_a (3-vectors) to the 4-point gradient / Hessian.
static void map_grad(int nvar, const double cm[][4], const double gv[][3], double* g) {
  for (int a = 0; a < 4; ++a)
    for (int d = 0; d < 3; ++d) {
      double s = 0;
      for (int m = 0; m < nvar; ++m) s += cm[m][a] * gv[m][d];
      g[3 * a + d] = s;
    }
}
// Hvv[m][n] is the 3x3 block d2f/du_m du_n.
static void map_hess(int nvar, const double cm[][4], const double Hvv[][3][9], double* H) {
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double s = 0;
          for (int m = 0; m < nvar; ++m)
            for (int n = 0; n < nvar; ++n) s += cm[m][a] * cm[n][b] * Hvv[m][n][3 * i + j];
          H[12 * (3 * a + i) + (3 * b + j)] = s;
        }
}

// point-point: s = |xa - xb|^2 ; slots ia, ib of the stencil.
static void dist_pp(const double* x, int ia, int ib, double* s, double* g, double* H) {
  double d[3];
  sub3(x + 3 * ia, x + 3 * ib, d);
  *s = dot3(d, d);
  if (!g) return;
  for (int i = 0; i < 12; ++i) g[i] = 0;
  for (int k = 0; k < 3; ++k) {
    g[3 * ia + k] = 2 * d[k];
    g[3 * ib + k] = -2 * d[k];
  }
  if (!H) return;
  for (int i = 0; i < 144; ++i) H[i] = 0;
  for (int k = 0; k < 3; ++k) {
    H[12 * (3 * ia + k) + 3 * ia + k] = 2;
    H[12 * (3 * ib + k) + 3 * ib + k] = 2;
    H[12 * (3 * ia + k) + 3 * ib + k] = -2;
    H[12 * (3 * ib + k) + 3 * ia + k] = -2;
  }
}

// point-line: s = |r|^2 - (r.e)^2 / (e.e), r = xp - x0, e = x1 - x0.
static void dist_pe(const double* x, int ip, int i0, int i1, double* s, double* g, double* H) {
  double r[3], e[3];
  sub3(x + 3 * ip, x + 3 * i0, r);
  sub3(x + 3 * i1, x + 3 * i0, e);
  double c = dot3(r, e), q = dot3(e, e);
  *s = dot3(r, r) - c * c / q;
  if (!g) return;
  double cm[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  cm[0][ip] = 1; cm[0][i0] = -1;   // r
  cm[1][i1] = 1; cm[1][i0] = -1;   // e
  double gv[2][3];
  for (int k = 0; k < 3; ++k) {
    gv[0][k] = 2 * r[k] - 2 * c * e[k] / q;
    gv[1][k] = -2 * c * r[k] / q + 2 * c * c * e[k] / (q * q);
  }
  map_grad(2, cm, gv, g);
  if (!H) return;
  double Hv[3][3][9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double dij = (i == j) ? 1.0 : 0.0;
      Hv[0][0][3 * i + j] = 2 * dij - 2 * e[i] * e[j] / q;
      Hv[0][1][3 * i + j] = -2 * (e[i] * r[j] + c * dij) / q + 4 * c * e[i] * e[j] / (q * q);
      Hv[1][1][3 * i + j] = -2 * r[i] * r[j] / q + 4 * c * (r[i] * e[j] + e[i] * r[j]) / (q * q) +
                            2 * c * c * dij / (q * q) - 8 * c * c * e[i] * e[j] / (q * q * q);
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Hv[1][0][3 * i + j] = Hv[0][1][3 * j + i];
  map_hess(2, cm, Hv, H);
}

// plane-type distance s = (v.n)^2 / (n.n), n = a x b, with v, a, b given as
// coefficient combinations of the stencil (point-plane and line-line).
static void dist_plane(const double* x, const double cm[3][4], double* s, double* g, double* H) {
  double v[3] = {0, 0, 0}, a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
  for (int k = 0; k < 4; ++k)
    for (int d = 0; d < 3; ++d) {
      v[d] += cm[0][k] * x[3 * k + d];
      a[d] += cm[1][k] * x[3 * k + d];
      b[d] += cm[2][k] * x[3 * k + d];
    }
  double n[3];
  cross3(a, b, n);
  double c = dot3(v, n), q = dot3(n, n);
  *s = c * c / q;
  if (!g) return;
  double gvv[3], gn[3];
  for (int k = 0; k < 3; ++k) {
    gvv[k] = 2 * c * n[k] / q;
    gn[k] = 2 * c * v[k] / q - 2 * c * c * n[k] / (q * q);
  }
  double gv[3][3];
  for (int k = 0; k < 3; ++k) gv[0][k] = gvv[k];
  cross3(b, gn, gv[1]);  // d/da = b x g_n
  cross3(gn, a, gv[2]);  // d/db = g_n x a
  map_grad(3, cm, gv, g);
  if (!H) return;
  double Gvv[9], Gvn[9], Gnn[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double dij = (i == j) ? 1.0 : 0.0;
      Gvv[3 * i + j] = 2 * n[i] * n[j] / q;
      Gvn[3 * i + j] = 2 * (n[i] * v[j] + c * dij) / q - 4 * c * n[i] * n[j] / (q * q);
      Gnn[3 * i + j] = 2 * v[i] * v[j] / q - 4 * c * (v[i] * n[j] + n[i] * v[j]) / (q * q) -
                       2 * c * c * dij / (q * q) + 8 * c * c * n[i] * n[j] / (q * q * q);
    }
  double Sa[9], Sb[9], Sg[9], mSb[9];
  skew(a, Sa);
  skew(b, Sb);
  skew(gn, Sg);
  for (int i = 0; i < 9; ++i) mSb[i] = -Sb[i];
  // dn/da = -[b]x, dn/db = [a]x
  double Hv[3][3][9], T[9], T2[9];
  std::memcpy(Hv[0][0], Gvv, sizeof(Gvv));
  matmul3(Gvn, mSb, Hv[0][1]);
  matmul3(Gvn, Sa, Hv[0][2]);
  matmul3(Sb, Gnn, T);  // (dn/da)^T = [b]x
  matmul3(T, mSb, Hv[1][1]);
  matmul3(T, Sa, T2);
  for (int i = 0; i < 9; ++i) Hv[1][2][i] = T2[i] - Sg[i];
  double mSa[9];
  for (int i = 0; i < 9; ++i) mSa[i] = -Sa[i];
  matmul3(mSa, Gnn, T);  // (dn/db)^T = -[a]x
  matmul3(T, Sa, Hv[2][2]);
  for (int m = 0; m < 3; ++m)
    for (int nn = 0; nn < m; ++nn)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Hv[m][nn][3 * i + j] = Hv[nn][m][3 * j + i];
  map_hess(3, cm, Hv, H);
}

// Point-triangle stencil (p, t0, t1, t2).  Types:
//   0,1,2: point-point with t0,t1,t2;  3,4,5: point-edge (t0t1),(t1t2),(t2t0);
//   6: point-plane (closest point inside the triangle).
void orc_pt_dist(const double* x, int type, double* s, double* g, double* H) {
  if (type <= 2) return dist_pp(x, 0, 1 + type, s, g, H);
  if (type <= 5) {
    int i0 = 1 + (type - 3), i1 = 1 + (type - 3 + 1) % 3;
    return dist_pe(x, 0, i0, i1, s, g, H);
  }
  const double cm[3][4] = {{1, -1, 0, 0}, {0, -1, 1, 0}, {0, -1, 0, 1}};
  dist_plane(x, cm, s, g, H);
}

// Edge-edge stencil (ea0, ea1, eb0, eb1).  Types:
//   0..3: point-point (ea0,eb0), (ea0,eb1), (ea1,eb0), (ea1,eb1);
//   4,5: point-edge eb0 / eb1 against edge a;  6,7: ea0 / ea1 against edge b;
//   8: line-line (closest points interior to both edges).
void orc_ee_dist(const double* x, int type, double* s, double* g, double* H) {
  switch (type) {
    case 0: return dist_pp(x, 0, 2, s, g, H);
    case 1: return dist_pp(x, 0, 3, s, g, H);
    case 2: return dist_pp(x, 1, 2, s, g, H);
    case 3: return dist_pp(x, 1, 3, s, g, H);
    case 4: return dist_pe(x, 2, 0, 1, s, g, H);
    case 5: return dist_pe(x, 3, 0, 1, s, g, H);
    case 6: return dist_pe(x, 0, 2, 3, s, g, H);
    case 7: return dist_pe(x, 1, 2, 3, s, g, H);
    default: {
      const double cm[3][4] = {{1, 0, -1, 0}, {-1, 1, 0, 0}, {0, 0, -1, 1}};
      dist_plane(x, cm, s, g, H);
    }
  }
}

// Point against segment (x0, x1): the segment parameter, clamped to [0, 1].
static double seg_param(const double* p, const double* x0, const double* x1) {
  double r[3], e[3];
  sub3(p, x0, r);
  sub3(x1, x0, e);
  double t = dot3(r, e) / dot3(e, e);
  return t < 0 ? 0.0 : (t > 1 ? 1.0 : t);
}

// Classify: the closest pair of points of the two primitives.  Returns the
// type; *s is that type's squared distance and w the closest-point weights,
// sum_k w_k x_k = (closest point on the first primitive) - (on the second).
int orc_pt_classify(const double* x, double* s_out, double* w) {
  const double *p = x, *t0 = x + 3, *t1 = x + 6, *t2 = x + 9;
  double a[3], b[3], v[3];
  sub3(t1, t0, a);
  sub3(t2, t0, b);
  sub3(p, t0, v);
  double aa = dot3(a, a), ab = dot3(a, b), bb = dot3(b, b), av = dot3(a, v), bv = dot3(b, v);
  double det = aa * bb - ab * ab;
  double b1 = (bb * av - ab * bv) / det, b2 = (aa * bv - ab * av) / det;
  if (b1 > 0 && b2 > 0 && b1 + b2 < 1) {
    orc_pt_dist(x, 6, s_out, nullptr, nullptr);
    w[0] = 1; w[1] = -(1 - b1 - b2); w[2] = -b1; w[3] = -b2;
    return 6;
  }
  int best = -1;
  double best_s = 0, best_t = 0;
  for (int k = 0; k < 3; ++k) {
    const double* e0 = x + 3 * (1 + k);
    const double* e1 = x + 3 * (1 + (k + 1) % 3);
    double t = seg_param(p, e0, e1);
    int type = (t == 0) ? k : (t == 1 ? (k + 1) % 3 : 3 + k);
    double s;
    orc_pt_dist(x, type, &s, nullptr, nullptr);
    if (best < 0 || s < best_s) { best = type; best_s = s; best_t = t; }
  }
  *s_out = best_s;
  w[0] = 1; w[1] = w[2] = w[3] = 0;
  if (best <= 2) w[1 + best] = -1;
  else {
    int k = best - 3;
    w[1 + k] = -(1 - best_t);
    w[1 + (k + 1) % 3] = -best_t;
  }
  return best;
}

int orc_ee_classify(const double* x, double* s_out, double* w) {
  const double *a0 = x, *a1 = x + 3, *b0 = x + 6, *b1 = x + 9;
  double u[3], v[3], r[3];
  sub3(a1, a0, u);
  sub3(b1, b0, v);
  sub3(a0, b0, r);
  double uu = dot3(u, u), uv = dot3(u, v), vv = dot3(v, v), ur = dot3(u, r), vr = dot3(v, r);
  double D = uu * vv - uv * uv;
  if (D > 1e-12 * uu * vv) {
    double sa = (uv * vr - vv * ur) / D, tb = (uu * vr - uv * ur) / D;
    if (sa > 0 && sa < 1 && tb > 0 && tb < 1) {
      orc_ee_dist(x, 8, s_out, nullptr, nullptr);
      w[0] = 1 - sa; w[1] = sa; w[2] = -(1 - tb); w[3] = -tb;
      return 8;
    }
  }
  // closest pair on the boundary of the parameter square: an endpoint against the other segment
  struct Cand { int pt, e0, e1; };
  const Cand cand[4] = {{2, 0, 1}, {3, 0, 1}, {0, 2, 3}, {1, 2, 3}};
  int best = -1;
  double best_s = 0, best_t = 0;
  int best_c = 0;
  for (int c = 0; c < 4; ++c) {
    double t = seg_param(x + 3 * cand[c].pt, x + 3 * cand[c].e0, x + 3 * cand[c].e1);
    int type;
    if (t > 0 && t < 1) type = 4 + c;
    else {
      int other = (t == 0) ? cand[c].e0 : cand[c].e1;
      int ia = cand[c].pt < 2 ? cand[c].pt : other;
      int ib = cand[c].pt < 2 ? other : cand[c].pt;
      type = 2 * ia + (ib - 2);
    }
    double s;
    orc_ee_dist(x, type, &s, nullptr, nullptr);
    if (best < 0 || s < best_s) { best = type; best_s = s; best_t = t; best_c = c; }
  }
  *s_out = best_s;
  w[0] = w[1] = w[2] = w[3] = 0;
  if (best <= 3) {
    w[best / 2] = 1;
    w[2 + best % 2] = -1;
  } else {
    const Cand& c = cand[best_c];
    double sg = c.pt < 2 ? 1.0 : -1.0;  // + on edge a, - on edge b
    w[c.pt] = sg;
    w[c.e0] = -sg * (1 - best_t);
    w[c.e1] = -sg * best_t;
  }
  return best;
}

// ---------------------------------------------------------------------------
// barrier and mollifier
// ---------------------------------------------------------------------------

// b(s) = -(s - sh)^2 ln(s / sh) for 0 < s < sh; derivatives w.r.t. s.
void orc_barrier(double s, double sh, double* b, double* b1, double* b2) {
  if (s >= sh) { *b = *b1 = *b2 = 0; return; }
  double d = s - sh, l = std::log(s / sh);
  *b = -d * d * l;
  *b1 = -(2 * d * l + d * d / s);
  *b2 = -(2 * l + 4 * d / s - d * d / (s * s));
}

// Edge-edge mollifier m(c), c = |(ea1-ea0) x (eb1-eb0)|^2.
void orc_ee_mollifier(const double* x, double eps_x, double* m, double* g, double* H) {
  double a[3], b[3], n[3];
  sub3(x + 3, x, a);
  sub3(x + 9, x + 6, b);
  cross3(a, b, n);
  double c = dot3(n, n);
  if (c >= eps_x) {
    *m = 1;
    if (g) for (int i = 0; i < 12; ++i) g[i] = 0;
    if (H) for (int i = 0; i < 144; ++i) H[i] = 0;
    return;
  }
  double r = c / eps_x;
  *m = -r * r + 2 * r;
  double m1 = (-2 * r + 2) / eps_x, m2 = -2 / (eps_x * eps_x);
  if (!g) return;
  const double cm[2][4] = {{-1, 1, 0, 0}, {0, 0, -1, 1}};
  double gc[2][3];
  cross3(b, n, gc[0]);
  cross3(n, a, gc[1]);
  for (int k = 0; k < 3; ++k) { gc[0][k] *= 2; gc[1][k] *= 2; }
  double gcs[12];
  map_grad(2, cm, gc, gcs);
  for (int i = 0; i < 12; ++i) g[i] = m1 * gcs[i];
  if (!H) return;
  double Sa[9], Sb[9], Sn[9], Hv[3][3][9];
  skew(a, Sa);
  skew(b, Sb);
  skew(n, Sn);
  double T[9];
  matmul3(Sb, Sb, T);
  for (int i = 0; i < 9; ++i) Hv[0][0][i] = -2 * T[i];
  matmul3(Sa, Sa, T);
  for (int i = 0; i < 9; ++i) Hv[1][1][i] = -2 * T[i];
  matmul3(Sb, Sa, T);
  for (int i = 0; i < 9; ++i) Hv[0][1][i] = 2 * T[i] - 2 * Sn[i];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Hv[1][0][3 * i + j] = Hv[0][1][3 * j + i];
  double Hc[144];
  map_hess(2, cm, Hv, Hc);
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) H[12 * i + j] = m2 * gcs[i] * gcs[j] + m1 * Hc[12 * i + j];
}

// One contact pair: kind 0 = point-triangle, 1 = edge-edge.
// E = kappa * m * b(s) (m = 1 for point-triangle), gradient, Hessian (optionally PSD-projected).
void orc_pair(int kind, int type, const double* x, double sh, double kappa, double eps_x, int project,
              double* E, double* g, double* H) {
  double s, gs[12], Hs[144];
  if (kind == 0) orc_pt_dist(x, type, &s, gs, Hs);
  else orc_ee_dist(x, type, &s, gs, Hs);
  double b, b1, b2;
  orc_barrier(s, sh, &b, &b1, &b2);
  double m = 1, gm[12], Hm[144];
  if (kind == 1) orc_ee_mollifier(x, eps_x, &m, gm, Hm);
  *E = kappa * m * b;
  for (int i = 0; i < 12; ++i) g[i] = kappa * (m * b1 * gs[i] + (kind == 1 ? b * gm[i] : 0.0));
  if (!H) return;
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) {
      double h = m * (b2 * gs[i] * gs[j] + b1 * Hs[12 * i + j]);
      if (kind == 1) h += b * Hm[12 * i + j] + b1 * (gm[i] * gs[j] + gs[i] * gm[j]);
      H[12 * i + j] = kappa * h;
    }
  if (project) orc_project_psd(12, H);
}

// ---------------------------------------------------------------------------
// lagged friction
// ---------------------------------------------------------------------------

// f0 and friends, eps = eps_v * dt:  f0(y) = -y^3/(3 eps^2) + y^2/eps + eps/3 (y < eps), y otherwise.
static double f0(double y, double eps) { return y < eps ? -y * y * y / (3 * eps * eps) + y * y / eps + eps / 3 : y; }
static double f1(double y, double eps) { return y < eps ? -y * y / (eps * eps) + 2 * y / eps : 1.0; }

// Friction on one lagged pair.  u = sum_k w_k (x_k - xt_k), P = I - n n^T,
// D = mu * lam * f0(|P u|).  Energy, gradient and Hessian (PSD by
// construction: eigenvalues f1(y)/y > 0 in the tangent plane orthogonal to
// P u, f1'(y) >= 0 along P u, 0 along n).
void orc_friction(const double* w, const double* n, double lam, double mu, double eps, const double* x,
                  const double* xt, double* E, double* g, double* H) {
  double u[3] = {0, 0, 0};
  for (int k = 0; k < 4; ++k)
    for (int d = 0; d < 3; ++d) u[d] += w[k] * (x[3 * k + d] - xt[3 * k + d]);
  double P[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P[3 * i + j] = (i == j ? 1.0 : 0.0) - n[i] * n[j];
  double t[3];
  for (int i = 0; i < 3; ++i) t[i] = P[3 * i] * u[0] + P[3 * i + 1] * u[1] + P[3 * i + 2] * u[2];
  double y = std::sqrt(dot3(t, t));
  double c = mu * lam;
  *E = c * f0(y, eps);
  // f1(y)/y, finite at y = 0
  double a = y < eps ? (-y / (eps * eps) + 2 / eps) : 1.0 / y;
  double gu[3];
  for (int i = 0; i < 3; ++i) gu[i] = c * a * t[i];
  for (int k = 0; k < 4; ++k)
    for (int d = 0; d < 3; ++d) g[3 * k + d] = w[k] * gu[d];
  if (!H) return;
  // d(a t)/du = a P + (da/dy) (t t^T) / y
  double Hu[9];
  double bcoef;
  if (y < eps) bcoef = (y > 0) ? (-1 / (eps * eps)) / y : 0.0;
  else bcoef = -1 / (y * y * y);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Hu[3 * i + j] = c * (a * P[3 * i + j] + bcoef * t[i] * t[j]);
  for (int k = 0; k < 4; ++k)
    for (int l = 0; l < 4; ++l)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[12 * (3 * k + i) + 3 * l + j] = w[k] * w[l] * Hu[3 * i + j];
}

// ---------------------------------------------------------------------------
// candidate pairs by brute force
// ---------------------------------------------------------------------------

// Scene topology for the contact routines.  Vertex ids index the global
// position array (FEM, then ABD surface, then kinematic vertices).
struct OrcSurf {
  int nsv, ntri, nedge;
  const int* sv;        // surface vertex ids
  const int* tri;       // 3 ids per triangle
  const int* edge;      // 2 ids per edge
  const int* vbody;     // body id of each vertex
  const int* bkind;     // kind of each body: 0 FEM, 1 ABD, 2 kinematic
};

static bool excluded(const OrcSurf& S, const int* va, int na, const int* vb, int nb) {
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j)
      if (va[i] == vb[j]) return true;
  int ba = S.vbody[va[0]], bb = S.vbody[vb[0]];
  int ka = S.bkind[ba], kb = S.bkind[bb];
  if (ba == bb && ka != 0) return true;  // same rigid (ABD or kinematic) body
  if (ka == 2 && kb == 2) return true;   // nothing free to move
  return false;
}

// All pairs with squared distance below sh.  Each output record holds
// kind (0 PT, 1 EE), primitive a, primitive b, type, 4 vertex ids, s.
// Returns the number of pairs (records beyond cap are not written).
struct PairRec { int r[8]; double s; };
static const int kChunks = 256;  // chunks of the outer loop index (output kept in chunk order)

int orc_active_pairs(const OrcSurf* Sp, const double* x, double sh, int cap, int* rec_i, double* rec_s) {
  const OrcSurf& S = *Sp;
  std::vector<std::vector<PairRec>> pt(kChunks), ee(kChunks);
#pragma omp parallel for schedule(dynamic, 1) num_threads(orc_get_threads())
  for (int c = 0; c < kChunks; ++c) {
    double xs[12], w[4], s;
    for (int i = (int)((long long)S.nsv * c / kChunks); i < (int)((long long)S.nsv * (c + 1) / kChunks); ++i) {
      int p = S.sv[i];
      for (int t = 0; t < S.ntri; ++t) {
        const int* tv = S.tri + 3 * t;
        if (excluded(S, &p, 1, tv, 3)) continue;
        int ids[4] = {p, tv[0], tv[1], tv[2]};
        for (int k = 0; k < 4; ++k)
          for (int d = 0; d < 3; ++d) xs[3 * k + d] = x[3 * ids[k] + d];
        int type = orc_pt_classify(xs, &s, w);
        if (s < sh) {
          PairRec q;
          q.r[0] = 0; q.r[1] = i; q.r[2] = t; q.r[3] = type;
          for (int k = 0; k < 4; ++k) q.r[4 + k] = ids[k];
          q.s = s;
          pt[c].push_back(q);
        }
      }
    }
    // edge-edge rows: chunk c takes the rows ea with ea mod kChunks == c (the triangular loop stays balanced)
    for (int ea = c; ea < S.nedge; ea += kChunks) {
      const int* va = S.edge + 2 * ea;
      for (int eb = ea + 1; eb < S.nedge; ++eb) {
        const int* vb = S.edge + 2 * eb;
        if (excluded(S, va, 2, vb, 2)) continue;
        int ids[4] = {va[0], va[1], vb[0], vb[1]};
        for (int k = 0; k < 4; ++k)
          for (int d = 0; d < 3; ++d) xs[3 * k + d] = x[3 * ids[k] + d];
        int type = orc_ee_classify(xs, &s, w);
        if (s < sh) {
          PairRec q;
          q.r[0] = 1; q.r[1] = ea; q.r[2] = eb; q.r[3] = type;
          for (int k = 0; k < 4; ++k) q.r[4 + k] = ids[k];
          q.s = s;
          ee[c].push_back(q);
        }
      }
    }
  }
  // serial order: point-triangle pairs by (vertex, triangle), then edge-edge pairs by (ea, eb)
  std::vector<const PairRec*> out;
  for (int c = 0; c < kChunks; ++c)
    for (const PairRec& q : pt[c]) out.push_back(&q);
  std::vector<const PairRec*> eev;
  for (int c = 0; c < kChunks; ++c)
    for (const PairRec& q : ee[c]) eev.push_back(&q);
  std::stable_sort(eev.begin(), eev.end(), [](const PairRec* a, const PairRec* b) {
    return a->r[1] != b->r[1] ? a->r[1] < b->r[1] : a->r[2] < b->r[2];
  });
  out.insert(out.end(), eev.begin(), eev.end());
  const int count = (int)out.size();
  for (int k = 0; k < count && k < cap; ++k) {
    for (int j = 0; j < 8; ++j) rec_i[8 * k + j] = out[k]->r[j];
    rec_s[k] = out[k]->s;
  }
  return count;
}

// ---------------------------------------------------------------------------
// additive CCD
// ---------------------------------------------------------------------------

static double pair_distance(int kind, const double* x) {
  double s, w[4];
  if (kind == 0) orc_pt_classify(x, &s, w);
  else orc_ee_classify(x, &s, w);
  return std::sqrt(s);
}

// Conservative time of impact in [0, tmax] for x + t p, stopping before the
// distance drops below s_frac times its start value.  The distance can shrink
// at most at rate lp (sum of the two primitives' largest relative speeds), so
// a step of (1 - s_frac) d0 / lp, and after that 0.9 d / lp, never skips a
// contact.  Returns tmax when no such approach happens within the step.
double orc_accd(int kind, const double* x0, const double* p0, double s_frac, double tmax, int max_iter) {
  double p[12], pbar[3] = {0, 0, 0};
  for (int k = 0; k < 4; ++k)
    for (int d = 0; d < 3; ++d) pbar[d] += 0.25 * p0[3 * k + d];
  for (int k = 0; k < 4; ++k)
    for (int d = 0; d < 3; ++d) p[3 * k + d] = p0[3 * k + d] - pbar[d];
  double nrm[4];
  for (int k = 0; k < 4; ++k) nrm[k] = std::sqrt(dot3(p + 3 * k, p + 3 * k));
  double lp = (kind == 0) ? nrm[0] + std::max(nrm[1], std::max(nrm[2], nrm[3]))
                          : std::max(nrm[0], nrm[1]) + std::max(nrm[2], nrm[3]);
  if (lp == 0) return tmax;
  double d0 = pair_distance(kind, x0);
  double target = s_frac * d0;
  double t = 0, tl = (1 - s_frac) * d0 / lp;
  double xt[12];
  for (int it = 0; it < max_iter; ++it) {
    double tn = t + tl;
    for (int i = 0; i < 12; ++i) xt[i] = x0[i] + tn * p[i];
    double d = pair_distance(kind, xt);
    // the first step keeps d >= target by the bound itself; only rounding could say otherwise
    if (d < target && it > 0) return t;
    t = tn;
    if (t >= tmax) return tmax;
    tl = 0.9 * d / lp;
  }
  return t;
}

static bool boxes_overlap(const double* lo_a, const double* hi_a, const double* lo_b, const double* hi_b) {
  for (int d = 0; d < 3; ++d)
    if (lo_a[d] > hi_b[d] || lo_b[d] > hi_a[d]) return false;
  return true;
}

static void swept_box(const double* x, const double* p, const int* ids, int n, double* lo, double* hi) {
  for (int d = 0; d < 3; ++d) { lo[d] = INFINITY; hi[d] = -INFINITY; }
  for (int k = 0; k < n; ++k)
    for (int d = 0; d < 3; ++d) {
      double a = x[3 * ids[k] + d], b = a + p[3 * ids[k] + d];
      lo[d] = std::min(lo[d], std::min(a, b));
      hi[d] = std::max(hi[d], std::max(a, b));
    }
}

// Largest step fraction alpha in (0, 1] along p: minimum ACCD time of impact
// over every pair whose swept boxes over [x, x + p] overlap.  The minimum and
// the candidate count do not depend on the order the pairs are visited in.
double orc_ccd_alpha(const OrcSurf* Sp, const double* x, const double* p, double s_frac, int max_iter,
                     int* n_cand) {
  const OrcSurf& S = *Sp;
  double alpha = 1.0;
  long long nc = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(orc_get_threads()) reduction(min : alpha) reduction(+ : nc)
  for (int c = 0; c < kChunks; ++c) {
    double xs[12], ps[12], la[3], ha[3], lb[3], hb[3];
    for (int i = (int)((long long)S.nsv * c / kChunks); i < (int)((long long)S.nsv * (c + 1) / kChunks); ++i) {
      int pv = S.sv[i];
      swept_box(x, p, &pv, 1, la, ha);
      for (int t = 0; t < S.ntri; ++t) {
        const int* tv = S.tri + 3 * t;
        if (excluded(S, &pv, 1, tv, 3)) continue;
        swept_box(x, p, tv, 3, lb, hb);
        if (!boxes_overlap(la, ha, lb, hb)) continue;
        int ids[4] = {pv, tv[0], tv[1], tv[2]};
        for (int k = 0; k < 4; ++k)
          for (int d = 0; d < 3; ++d) { xs[3 * k + d] = x[3 * ids[k] + d]; ps[3 * k + d] = p[3 * ids[k] + d]; }
        ++nc;
        alpha = std::min(alpha, orc_accd(0, xs, ps, s_frac, 1.0, max_iter));
      }
    }
    for (int ea = c; ea < S.nedge; ea += kChunks) {
      const int* va = S.edge + 2 * ea;
      swept_box(x, p, va, 2, la, ha);
      for (int eb = ea + 1; eb < S.nedge; ++eb) {
        const int* vb = S.edge + 2 * eb;
        if (excluded(S, va, 2, vb, 2)) continue;
        swept_box(x, p, vb, 2, lb, hb);
        if (!boxes_overlap(la, ha, lb, hb)) continue;
        int ids[4] = {va[0], va[1], vb[0], vb[1]};
        for (int k = 0; k < 4; ++k)
          for (int d = 0; d < 3; ++d) { xs[3 * k + d] = x[3 * ids[k] + d]; ps[3 * k + d] = p[3 * ids[k] + d]; }
        ++nc;
        alpha = std::min(alpha, orc_accd(1, xs, ps, s_frac, 1.0, max_iter));
      }
    }
  }
  if (n_cand) *n_cand = (int)nc;
  return alpha;
}

// ---------------------------------------------------------------------------
// affine body orthogonality energy (§III-C.1, "stiff orthogonality energy")
// ---------------------------------------------------------------------------

// E = k * sum_ij (a_i . a_j - delta_ij)^2 over the columns a_i of A
// (a = [a_0, a_1, a_2], 9 values), gradient and 9x9 Hessian.
void orc_abd_orth(const double* a, double k, int project, double* E, double* g, double* H) {
  double G[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G[3 * i + j] = dot3(a + 3 * i, a + 3 * j) - (i == j ? 1.0 : 0.0);
  double e = 0;
  for (int i = 0; i < 9; ++i) e += G[i] * G[i];
  *E = k * e;
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) {
      double s = 0;
      for (int j = 0; j < 3; ++j) s += G[3 * i + j] * a[3 * j + d];
      g[3 * i + d] = 4 * k * s;
    }
  if (!H) return;
  double AAt[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int j = 0; j < 3; ++j) s += a[3 * j + r] * a[3 * j + c];
      AAt[3 * r + c] = s;
    }
  for (int ki = 0; ki < 3; ++ki)
    for (int li = 0; li < 3; ++li)
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          double h = a[3 * li + r] * a[3 * ki + c] + (r == c ? G[3 * ki + li] : 0.0);
          if (ki == li) h += AAt[3 * r + c];
          H[9 * (3 * ki + r) + 3 * li + c] = 4 * k * h;
        }
  if (project) orc_project_psd(9, H);
}

}  // extern "C"
