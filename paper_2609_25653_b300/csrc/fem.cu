// Per-node and per-element kernels of the incremental potential (Eq. 3):
// predictor, kinematic targets, vertex positions, inertia, Neo-Hookean
// elasticity (§III-C.1), stitch springs (Eq. 2), affine-body orthogonality,
// step update and velocities.
#include <type_traits>
#include "common.cuh"
#include "eig.cuh"
#include "kernels.h"

namespace ipc {

// z_t <- z ; z~ = z + dt zd + dt^2 a, a = gravity on FEM nodes and on ABD translation nodes.
__global__ void k_predict(int n_nodes, int nf, const double* __restrict__ z, const double* __restrict__ zd, double dt,
                          d3 g, double* __restrict__ z_t, double* __restrict__ z_tilde) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  bool grav = (i < nf) || ((i - nf) % 4 == 0);
  double dt2 = dt * dt;
  for (int d = 0; d < 3; ++d) {
    double zi = z[3 * i + d];
    z_t[3 * i + d] = zi;
    z_tilde[3 * i + d] = zi + dt * zd[3 * i + d] + (grav ? dt2 * comp(g, d) : 0.0);
  }
}

// x = R xbar + t for every kinematic vertex; stitch anchors likewise.
__global__ void k_kin_targets(DevScene S, const double* __restrict__ T, double* __restrict__ xk_hat,
                              double* __restrict__ stitch_hat) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < S.nk) {
    int b = S.kin_vbody[i];
    const double* M = T + 12 * b;
    d3 xb = ld3(S.xbar, S.nf + S.na_v + i);
    st3(xk_hat, i, mk(M[0] * xb.x + M[1] * xb.y + M[2] * xb.z + M[3], M[4] * xb.x + M[5] * xb.y + M[6] * xb.z + M[7],
                      M[8] * xb.x + M[9] * xb.y + M[10] * xb.z + M[11]));
  }
  if (i < S.n_stitch) {
    const double* M = T + 12 * S.stitch_b[i];
    d3 xb = ld3(S.stitch_X, i);
    st3(stitch_hat, i, mk(M[0] * xb.x + M[1] * xb.y + M[2] * xb.z + M[3], M[4] * xb.x + M[5] * xb.y + M[6] * xb.z + M[7],
                          M[8] * xb.x + M[9] * xb.y + M[10] * xb.z + M[11]));
  }
}

// All vertex positions from the DOFs and the kinematic positions.
__global__ void k_vertex_positions(DevScene S, const double* __restrict__ z, const double* __restrict__ xk,
                                   double* __restrict__ xv) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= S.nv) return;
  int k = S.vkind[v];
  d3 x;
  if (k == VK_FEM) x = ld3(z, v);
  else if (k == VK_ABD) {
    int base = S.nf + 4 * S.vabd[v];
    d3 xb = ld3(S.xbar, v);
    x = ld3(z, base) + xb.x * ld3(z, base + 1) + xb.y * ld3(z, base + 2) + xb.z * ld3(z, base + 3);
  } else x = ld3(xk, v - S.nf - S.na_v);
  st3(xv, v, x);
}

// Vertex displacement of a Newton direction: FEM p, ABD J(xbar) p, kinematic p_D.
__global__ void k_vertex_disp(DevScene S, const double* __restrict__ p, const double* __restrict__ pD,
                              double* __restrict__ pv) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= S.nv) return;
  int k = S.vkind[v];
  d3 x;
  if (k == VK_FEM) x = ld3(p, v);
  else if (k == VK_ABD) {
    int base = S.nf + 4 * S.vabd[v];
    d3 xb = ld3(S.xbar, v);
    x = ld3(p, base) + xb.x * ld3(p, base + 1) + xb.y * ld3(p, base + 2) + xb.z * ld3(p, base + 3);
  } else x = ld3(pD, v - S.nf - S.na_v);
  st3(pv, v, x);
}

// Inertia 1/2 (z - z~)^T M (z - z~): energy into E[0]; gradient M (z - z~) added into g.
__global__ void k_inertia(DevScene S, const double* __restrict__ z, const double* __restrict__ z_tilde,
                          acc_t* __restrict__ g, acc_t* __restrict__ E, int want_grad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < S.nf) {
    d3 dz = ld3(z, i) - ld3(z_tilde, i);
    double m = S.node_mass[i];
    e = 0.5 * m * dot(dz, dz);
    if (S.E_sc) scene_energy(S, S.node_scene[i], 0, e);
    if (want_grad) acc_add3(g, i, m * dz, S.err);
  } else if (i < S.n_nodes) {
    int b = (i - S.nf) / 4, r = (i - S.nf) % 4;
    int base = S.nf + 4 * b;
    const double* Sm = S.abd_S + 16 * b;
    d3 acc = mk(0, 0, 0);
    for (int s = 0; s < 4; ++s) acc = acc + Sm[4 * r + s] * (ld3(z, base + s) - ld3(z_tilde, base + s));
    e = 0.5 * dot(ld3(z, i) - ld3(z_tilde, i), acc);
    if (S.E_sc) scene_energy(S, S.node_scene[i], 0, e);
    if (want_grad) acc_add3(g, i, acc, S.err);
  }
  double s = block_sum(e);
  if (threadIdx.x == 0) acc_add(E, s, S.err);
}


// ---------------------------------------------------------------------------
// analytic PSD projection of the Neo-Hookean Hessian
// ---------------------------------------------------------------------------
// With a rotation-variant SVD F = U diag(s) V^T (U, V rotations, s_2 may be
// negative) the second derivative of J = det F in the rotated frame
// X = U^T dF V is the quadratic form sum_{i<j} s_k (X_ii X_jj - X_ij X_ji)
// (k the third index), and cof F = U diag(s1 s2, s0 s2, s0 s1) V^T.  Hence
// d2Psi/dF2 = mu I + lam g g^T + kJ d2J/dF2 has the eigenvectors
//   twist_k = U (e_i e_j^T - e_j e_i^T) V^T / sqrt2,  eigenvalue mu + kJ s_k
//   flip_k  = U (e_i e_j^T + e_j e_i^T) V^T / sqrt2,  eigenvalue mu - kJ s_k
// and three in span{U e_m e_m^T V^T} from the 3x3 matrix
//   A = mu I + lam c c^T + kJ [[0, s2, s1], [s2, 0, s0], [s1, s0, 0]],
//   c = (s1 s2, s0 s2, s0 s1).
// Keeping the non-negative eigenvalues gives the nearest PSD matrix.

// cyclic Jacobi for a symmetric 3x3 (row-major); eigenvectors in the columns of V
__device__ inline void jacobi3(double* A, double* V) {
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 24; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    double tot = A[0] * A[0] + A[4] * A[4] + A[8] * A[8] + 2.0 * off;
    if (off <= 1e-32 * tot || tot == 0.0) break;
    const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
    for (int r = 0; r < 3; ++r) {
      int p = P[r], q = Q[r];
      double apq = A[3 * p + q];
      if (apq == 0.0) continue;
      double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
      double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
      for (int k = 0; k < 3; ++k) {
        double akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = c * akp - sn * akq;
        A[3 * k + q] = sn * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        double apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = c * apk - sn * aqk;
        A[3 * q + k] = sn * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        double vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - sn * vkq;
        V[3 * k + q] = sn * vkp + c * vkq;
      }
    }
  }
}

// F = U diag(s) V^T with U, V proper rotations (columns), s0 >= s1 >= |s2|, s2 signed.
__device__ inline void svd3_rv(const d3* f, d3* U, d3* Vc, double* s) {
  // columns f[j] of F; S = F^T F
  double A[9], V[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[3 * i + j] = dot(f[i], f[j]);
  jacobi3(A, V);
  double e[3] = {A[0], A[4], A[8]};
  int ord[3] = {0, 1, 2};
  for (int a = 0; a < 2; ++a)
    for (int b = a + 1; b < 3; ++b)
      if (e[ord[b]] > e[ord[a]]) { int t = ord[a]; ord[a] = ord[b]; ord[b] = t; }
  for (int m = 0; m < 3; ++m) Vc[m] = mk(V[ord[m]], V[3 + ord[m]], V[6 + ord[m]]);
  if (dot(cross(Vc[0], Vc[1]), Vc[2]) < 0.0) Vc[2] = -1.0 * Vc[2];
  // b_m = F v_m = sum_j v_m[j] f_j
  d3 b[3];
  for (int m = 0; m < 3; ++m) b[m] = Vc[m].x * f[0] + Vc[m].y * f[1] + Vc[m].z * f[2];
  double n0 = sqrt(dot(b[0], b[0]));
  U[0] = n0 > 1e-300 ? (1.0 / n0) * b[0] : mk(1, 0, 0);
  d3 u1 = b[1] - dot(U[0], b[1]) * U[0];
  double n1 = sqrt(dot(u1, u1));
  if (n1 > 1e-14 * (n0 + 1e-300)) u1 = (1.0 / n1) * u1;
  else {
    d3 t = fabs(U[0].x) < 0.9 ? mk(1, 0, 0) : mk(0, 1, 0);
    u1 = cross(U[0], t);
    u1 = (1.0 / sqrt(dot(u1, u1))) * u1;
  }
  U[1] = u1;
  U[2] = cross(U[0], U[1]);
  s[0] = dot(U[0], b[0]);
  s[1] = dot(U[1], b[1]);
  s[2] = dot(U[2], b[2]);
}

// Projected 12x12 tet Hessian (row-major, times sv) from the eigen-modes above.
// Cc[a][j]: dF(:,j)/dx_a coefficients.
__device__ inline void snh_projected_hessian(const d3* f, double mu, double lam, const double Cc[4][3], double sv,
                                             double* H12) {
  d3 U[3], V[3];
  double s[3];
  svd3_rv(f, U, V, s);
  double J = s[0] * s[1] * s[2];
  double kJ = lam * (J - 1.0) - mu;
  for (int i = 0; i < 144; ++i) H12[i] = 0.0;
  // w_a = M C[a], M = U B V^T  =>  M c = U (B (V^T c))
  double Vt_c[4][3];
  for (int a = 0; a < 4; ++a)
    for (int m = 0; m < 3; ++m) Vt_c[a][m] = V[m].x * Cc[a][0] + V[m].y * Cc[a][1] + V[m].z * Cc[a][2];
  auto add_mode = [&](const double* B, double lamb) {
    if (!(lamb > 0.0)) return;
    double w[12];
    for (int a = 0; a < 4; ++a) {
      double y0 = B[0] * Vt_c[a][0] + B[1] * Vt_c[a][1] + B[2] * Vt_c[a][2];
      double y1 = B[3] * Vt_c[a][0] + B[4] * Vt_c[a][1] + B[5] * Vt_c[a][2];
      double y2 = B[6] * Vt_c[a][0] + B[7] * Vt_c[a][1] + B[8] * Vt_c[a][2];
      d3 m = y0 * U[0] + y1 * U[1] + y2 * U[2];
      w[3 * a] = m.x; w[3 * a + 1] = m.y; w[3 * a + 2] = m.z;
    }
    double c = sv * lamb;
    for (int i = 0; i < 12; ++i) {  // upper triangle; the lower one is its mirror
      double ci = c * w[i];
      for (int j = i; j < 12; ++j) H12[12 * i + j] += ci * w[j];
    }
  };
  const double r2 = 0.70710678118654752440;
  const int PI[3] = {1, 0, 0}, PJ[3] = {2, 2, 1};  // pair (i, j) for k = 0, 1, 2
  for (int k = 0; k < 3; ++k) {
    int i = PI[k], j = PJ[k];
    double B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    B[3 * i + j] = r2; B[3 * j + i] = -r2;
    add_mode(B, mu + kJ * s[k]);   // twist
    B[3 * j + i] = r2;
    add_mode(B, mu - kJ * s[k]);   // flip
  }
  double c3[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};
  double A[9], Y[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[3 * i + j] = (i == j ? mu : 0.0) + lam * c3[i] * c3[j];
  A[1] += kJ * s[2]; A[3] += kJ * s[2];
  A[2] += kJ * s[1]; A[6] += kJ * s[1];
  A[5] += kJ * s[0]; A[7] += kJ * s[0];
  jacobi3(A, Y);
  for (int q = 0; q < 3; ++q) {
    double B[9] = {Y[q], 0, 0, 0, Y[3 + q], 0, 0, 0, Y[6 + q]};
    add_mode(B, A[4 * q]);
  }
  for (int i = 1; i < 12; ++i)
    for (int j = 0; j < i; ++j) H12[12 * i + j] = H12[12 * j + i];
}

// The same projection in FP32, for the mixed-precision path (whose operator is
// applied in FP32 anyway): the FP64 pipe of this part issues 2 FMA per clock
// per SM and this projection is ~3k FMA per tet; the FP32 pipe issues 128.
__device__ inline void jacobi3f(float* A, float* V) {
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.f : 0.f;
  for (int sweep = 0; sweep < 16; ++sweep) {
    float off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    float tot = A[0] * A[0] + A[4] * A[4] + A[8] * A[8] + 2.f * off;
    if (off <= 1e-14f * tot || tot == 0.f) break;
    const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
    for (int r = 0; r < 3; ++r) {
      int p = P[r], q = Q[r];
      float apq = A[3 * p + q];
      if (apq == 0.f) continue;
      float theta = (A[3 * q + q] - A[3 * p + p]) / (2.f * apq);
      float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
      float c = 1.f / sqrtf(t * t + 1.f), sn = t * c;
      for (int k = 0; k < 3; ++k) {
        float akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = c * akp - sn * akq;
        A[3 * k + q] = sn * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        float apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = c * apk - sn * aqk;
        A[3 * q + k] = sn * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        float vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - sn * vkq;
        V[3 * k + q] = sn * vkp + c * vkq;
      }
    }
  }
}

__device__ inline float dotf3(const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ inline void crossf3(const float* a, const float* b, float* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// FP32 counterpart of snh_projected_hessian (same modes and eigenvalues).
__device__ inline void snh_projected_hessian_f32(const d3* fd, double mu_d, double lam_d, const double Cc_d[4][3],
                                                 double sv_d, float* H12) {
  float f[3][3];
  for (int j = 0; j < 3; ++j) { f[j][0] = (float)fd[j].x; f[j][1] = (float)fd[j].y; f[j][2] = (float)fd[j].z; }
  const float mu = (float)mu_d, lam = (float)lam_d, sv = (float)sv_d;
  float Cc[4][3];
  for (int a = 0; a < 4; ++a)
    for (int j = 0; j < 3; ++j) Cc[a][j] = (float)Cc_d[a][j];
  // rotation-variant SVD F = U diag(s) V^T from the eigen-decomposition of F^T F
  float A[9], Vm[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[3 * i + j] = dotf3(f[i], f[j]);
  jacobi3f(A, Vm);
  float e[3] = {A[0], A[4], A[8]};
  int ord[3] = {0, 1, 2};
  for (int a = 0; a < 2; ++a)
    for (int b = a + 1; b < 3; ++b)
      if (e[ord[b]] > e[ord[a]]) { int t = ord[a]; ord[a] = ord[b]; ord[b] = t; }
  float V[3][3];
  for (int m = 0; m < 3; ++m) { V[m][0] = Vm[ord[m]]; V[m][1] = Vm[3 + ord[m]]; V[m][2] = Vm[6 + ord[m]]; }
  float c01[3];
  crossf3(V[0], V[1], c01);
  if (dotf3(c01, V[2]) < 0.f) { V[2][0] = -V[2][0]; V[2][1] = -V[2][1]; V[2][2] = -V[2][2]; }
  float bvec[3][3];
  for (int m = 0; m < 3; ++m)
    for (int d = 0; d < 3; ++d) bvec[m][d] = V[m][0] * f[0][d] + V[m][1] * f[1][d] + V[m][2] * f[2][d];
  float U[3][3];
  const float n0 = sqrtf(dotf3(bvec[0], bvec[0]));
  for (int d = 0; d < 3; ++d) U[0][d] = n0 > 1e-30f ? bvec[0][d] / n0 : (d == 0 ? 1.f : 0.f);
  float u1[3];
  const float pr = dotf3(U[0], bvec[1]);
  for (int d = 0; d < 3; ++d) u1[d] = bvec[1][d] - pr * U[0][d];
  const float n1 = sqrtf(dotf3(u1, u1));
  if (n1 > 1e-6f * (n0 + 1e-30f)) {
    for (int d = 0; d < 3; ++d) u1[d] /= n1;
  } else {
    float t[3] = {fabsf(U[0][0]) < 0.9f ? 1.f : 0.f, fabsf(U[0][0]) < 0.9f ? 0.f : 1.f, 0.f};
    crossf3(U[0], t, u1);
    const float nn = sqrtf(dotf3(u1, u1));
    for (int d = 0; d < 3; ++d) u1[d] /= nn;
  }
  for (int d = 0; d < 3; ++d) U[1][d] = u1[d];
  crossf3(U[0], U[1], U[2]);
  const float s[3] = {dotf3(U[0], bvec[0]), dotf3(U[1], bvec[1]), dotf3(U[2], bvec[2])};
  const float J = s[0] * s[1] * s[2];
  const float kJ = lam * (J - 1.f) - mu;
  for (int i = 0; i < 144; ++i) H12[i] = 0.f;
  float Vt_c[4][3];
  for (int a = 0; a < 4; ++a)
    for (int m = 0; m < 3; ++m) Vt_c[a][m] = V[m][0] * Cc[a][0] + V[m][1] * Cc[a][1] + V[m][2] * Cc[a][2];
  auto add_mode = [&](const float* B, float lamb) {
    if (!(lamb > 0.f)) return;
    float w[12];
    for (int a = 0; a < 4; ++a) {
      const float y0 = B[0] * Vt_c[a][0] + B[1] * Vt_c[a][1] + B[2] * Vt_c[a][2];
      const float y1 = B[3] * Vt_c[a][0] + B[4] * Vt_c[a][1] + B[5] * Vt_c[a][2];
      const float y2 = B[6] * Vt_c[a][0] + B[7] * Vt_c[a][1] + B[8] * Vt_c[a][2];
      for (int d = 0; d < 3; ++d) w[3 * a + d] = y0 * U[0][d] + y1 * U[1][d] + y2 * U[2][d];
    }
    const float c = sv * lamb;
    for (int i = 0; i < 12; ++i) {  // upper triangle; the lower one is its mirror
      const float ci = c * w[i];
      for (int j = i; j < 12; ++j) H12[12 * i + j] += ci * w[j];
    }
  };
  const float r2 = 0.70710678f;
  const int PI[3] = {1, 0, 0}, PJ[3] = {2, 2, 1};
  for (int k = 0; k < 3; ++k) {
    const int i = PI[k], j = PJ[k];
    float B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    B[3 * i + j] = r2; B[3 * j + i] = -r2;
    add_mode(B, mu + kJ * s[k]);
    B[3 * j + i] = r2;
    add_mode(B, mu - kJ * s[k]);
  }
  const float c3[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};
  float Am[9], Y[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Am[3 * i + j] = (i == j ? mu : 0.f) + lam * c3[i] * c3[j];
  Am[1] += kJ * s[2]; Am[3] += kJ * s[2];
  Am[2] += kJ * s[1]; Am[6] += kJ * s[1];
  Am[5] += kJ * s[0]; Am[7] += kJ * s[0];
  jacobi3f(Am, Y);
  for (int q = 0; q < 3; ++q) {
    const float B[9] = {Y[q], 0, 0, 0, Y[3 + q], 0, 0, 0, Y[6 + q]};
    add_mode(B, Am[4 * q]);
  }
  for (int i = 1; i < 12; ++i)
    for (int j = 0; j < i; ++j) H12[12 * i + j] = H12[12 * j + i];
}

// Neo-Hookean energy Psi = mu/2 (|F|^2 - 3) - mu (J - 1) + lam/2 (J - 1)^2 per tet (§III-C.1),
// its gradient and PSD-projected Hessian scattered into the BSR matrix.
// scale = dt^2 for the incremental potential; mode: 0 energy only, 1 + gradient, 2 + Hessian.
// F32H: the projected Hessian in FP32 (mixed precision); energy and gradient always FP64.
// Outputs: g (accumulators) or tG (the tet's 12 gradient entries, per tet); tU (the upper triangle of
// the tet's 12x12, 78 values per tet, row by row) and/or tetH (the full 12x12, per tet).
template <bool F32H>
__global__ void __launch_bounds__(128) k_elastic(DevScene S, const double* __restrict__ xv, double scale, int mode,
                                                 int project, acc_t* __restrict__ g, double* __restrict__ tG,
                                                 double* __restrict__ tU, double* __restrict__ tetH,
                                                 acc_t* __restrict__ E) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  double energy = 0.0;
  if (e < S.nt) {
    int4 t = S.tets[e];
    int id[4] = {t.x, t.y, t.z, t.w};
    d3 x0 = ld3(xv, id[0]);
    d3 c1 = ld3(xv, id[1]) - x0, c2 = ld3(xv, id[2]) - x0, c3 = ld3(xv, id[3]) - x0;
    const double* B = S.B + 9 * e;
    // F = Ds B, columns f_j = sum_k Ds(:,k) B(k,j)
    d3 f[3];
    for (int j = 0; j < 3; ++j) f[j] = B[j] * c1 + B[3 + j] * c2 + B[6 + j] * c3;
    d3 cf[3] = {cross(f[1], f[2]), cross(f[2], f[0]), cross(f[0], f[1])};
    double J = dot(f[0], cf[0]);
    double Ic = dot(f[0], f[0]) + dot(f[1], f[1]) + dot(f[2], f[2]);
    double mu = S.mu[e], lam = S.lam[e], V = S.vol[e];
    energy = V * (0.5 * mu * (Ic - 3.0) - mu * (J - 1.0) + 0.5 * lam * (J - 1.0) * (J - 1.0));
    if (S.E_sc) scene_energy(S, scene_of_vertex(S, id[0]), 1, energy);
    if (mode >= 1) {
      double kJ = lam * (J - 1.0) - mu;
      d3 Pc[3];  // columns of P
      for (int j = 0; j < 3; ++j) Pc[j] = mu * f[j] + kJ * cf[j];
      double Cc[4][3];
      for (int j = 0; j < 3; ++j) {
        Cc[1][j] = B[j];
        Cc[2][j] = B[3 + j];
        Cc[3][j] = B[6 + j];
        Cc[0][j] = -(B[j] + B[3 + j] + B[6 + j]);
      }
      double sv = scale * V;
      for (int a = 0; a < 4; ++a) {
        d3 ga = Cc[a][0] * Pc[0] + Cc[a][1] * Pc[1] + Cc[a][2] * Pc[2];
        if (g) acc_add3(g, id[a], sv * ga, S.err);
        if (tG) {
          tG[12 * (size_t)e + 3 * a] = sv * ga.x;
          tG[12 * (size_t)e + 3 * a + 1] = sv * ga.y;
          tG[12 * (size_t)e + 3 * a + 2] = sv * ga.z;
        }
      }
      if (mode >= 2 && project) {
        using HC = typename std::conditional<F32H, float, double>::type;
        HC H12[144];
        if constexpr (F32H) snh_projected_hessian_f32(f, mu, lam, Cc, sv, H12);
        else snh_projected_hessian(f, mu, lam, Cc, sv, H12);
        if (tU) {
          double* u = tU + 78 * (size_t)e;
          for (int r = 0, o = 0; r < 12; ++r)
            for (int c = r; c < 12; ++c) u[o++] = (double)H12[12 * r + c];
        }
        if (tetH)
          for (int i = 0; i < 144; ++i) tetH[144 * (size_t)e + i] = (double)H12[i];
      } else if (mode >= 2) {
        double H[81];
        double gv[9] = {cf[0].x, cf[0].y, cf[0].z, cf[1].x, cf[1].y, cf[1].z, cf[2].x, cf[2].y, cf[2].z};
        for (int p = 0; p < 9; ++p)
          for (int q = 0; q < 9; ++q) H[9 * p + q] = (p == q ? mu : 0.0) + lam * gv[p] * gv[q];
        // d2J/df_a df_b blocks: (0,1) = -[f2]x, (0,2) = [f1]x, (1,2) = -[f0]x
        const int A_[3] = {0, 0, 1}, B_[3] = {1, 2, 2}, W_[3] = {2, 1, 0};
        const double sg[3] = {-1.0, 1.0, -1.0};
        for (int k = 0; k < 3; ++k) {
          d3 w = f[W_[k]];
          double Sk[9] = {0, -w.z, w.y, w.z, 0, -w.x, -w.y, w.x, 0};
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
              double v = kJ * sg[k] * Sk[3 * i + j];
              H[9 * (3 * A_[k] + i) + 3 * B_[k] + j] += v;
              H[9 * (3 * B_[k] + j) + 3 * A_[k] + i] += v;
            }
        }
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            double blk[9];
            for (int i = 0; i < 3; ++i)
              for (int k = 0; k < 3; ++k) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j)
                  for (int l = 0; l < 3; ++l) s += Cc[a][j] * Cc[b][l] * H[9 * (3 * j + i) + 3 * l + k];
                blk[3 * i + k] = sv * s;
              }
            // upper triangle of the tet's 12x12: rows 3a + i <= columns 3b + k
            if (tU)
              for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) {
                  const int r = 3 * a + i, c = 3 * b + k;
                  if (r <= c) tU[78 * (size_t)e + 12 * r - r * (r - 1) / 2 + (c - r)] = blk[3 * i + k];
                }
            if (tetH)
              for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) tetH[144 * (size_t)e + 12 * (3 * a + i) + 3 * b + k] = blk[3 * i + k];
          }
      }
    }
  }
  double s = block_sum(energy);
  if (threadIdx.x == 0 && E) acc_add(E, s, S.err);
}

// Stitch springs 1/2 k_c |x_i - x^_i|^2 (Eq. 2); the constant Hessian k_c I is part of the fixed matrix.
__global__ void k_stitch(DevScene S, const double* __restrict__ xv, const double* __restrict__ stitch_hat, double k_c_unused,
                         double scale, int mode, acc_t* __restrict__ g, acc_t* __restrict__ E) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < S.n_stitch) {
    int v = S.stitch_v[i];
    const double k_c = S.scene_kc[scene_of_vertex(S, v)];
    d3 d = ld3(xv, v) - ld3(stitch_hat, i);
    e = 0.5 * k_c * dot(d, d);
    if (S.E_sc) scene_energy(S, scene_of_vertex(S, v), 4, e);
    if (mode >= 1) acc_add3(g, v, (scale * k_c) * d, S.err);
  }
  double s = block_sum(e);
  if (threadIdx.x == 0) acc_add(E, s, S.err);
}

// ABD orthogonality kappa_A V sum_ij (a_i . a_j - delta_ij)^2 over the columns of A.
__global__ void k_abd_orth(DevScene S, const double* __restrict__ z, double kappa_A, double scale, int mode, int project,
                           acc_t* __restrict__ g, acc_t* __restrict__ Hval, acc_t* __restrict__ E) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (b < S.nab) {
    int base = S.nf + 4 * b;
    d3 a[3] = {ld3(z, base + 1), ld3(z, base + 2), ld3(z, base + 3)};
    double k = kappa_A * S.abd_vol[b];
    double G[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) G[i][j] = dot(a[i], a[j]) - (i == j ? 1.0 : 0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) e += G[i][j] * G[i][j];
    e *= k;
    if (S.E_sc) scene_energy(S, S.node_scene[base], 5, e);
    if (mode >= 1) {
      for (int i = 0; i < 3; ++i) {
        d3 gi = 4.0 * k * (G[i][0] * a[0] + G[i][1] * a[1] + G[i][2] * a[2]);
        acc_add3(g, base + 1 + i, scale * gi, S.err);
      }
    }
    if (mode >= 2) {
      double H[81];
      double AAt[9];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) AAt[3 * r + c] = comp(a[0], r) * comp(a[0], c) + comp(a[1], r) * comp(a[1], c) +
                                                     comp(a[2], r) * comp(a[2], c);
      for (int ki = 0; ki < 3; ++ki)
        for (int li = 0; li < 3; ++li)
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
              double h = comp(a[li], r) * comp(a[ki], c) + (r == c ? G[ki][li] : 0.0);
              if (ki == li) h += AAt[3 * r + c];
              H[9 * (3 * ki + r) + 3 * li + c] = 4.0 * k * h;
            }
      if (project) project_psd<9, double>(H);
      for (int ki = 0; ki < 3; ++ki)
        for (int li = 0; li < 3; ++li) {
          acc_t* dst = Hval + 27 * (size_t)S.abd_blk[16 * b + 4 * (1 + ki) + (1 + li)];
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) acc_add(dst + 3 * (3 * r + c), scale * H[9 * (3 * ki + r) + 3 * li + c], S.err);
        }
    }
  }
  double s = block_sum(e);
  if (threadIdx.x == 0) acc_add(E, s, S.err);
}

// Joint drive potentials (E_joint of Eq. 3), one thread per joint.  Side a
// enters with sign +, side b with sign -; a side's map to world is
// w . (p, a0, a1, a2) with weights w = (1, v) for a body-frame point v and
// (0, v) for a direction, so the residual is r = sum_m w_m q_m - t over the
// eight pseudo-nodes of the two bodies (the world side has none).  Energy
// k/2 |r|^2, gradient k w_m r at pseudo-node m, Hessian k w_m w_n I for the
// block pair (m, n): constant in z and positive semi-definite, so nothing is
// projected.
__global__ void k_joints(DevScene S, const double* __restrict__ z, double scale, int mode, acc_t* __restrict__ g,
                         acc_t* __restrict__ Hval, acc_t* __restrict__ E) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (j < S.nj) {
    double w[8];
    int node[8];
    d3 r = {-S.jt_t[3 * j], -S.jt_t[3 * j + 1], -S.jt_t[3 * j + 2]};
    for (int s = 0; s < 2; ++s) {
      const int b = S.jt_body[2 * j + s];
      const d3 v = ld3(s == 0 ? S.jt_va : S.jt_vb, j);
      const double sg = s == 0 ? 1.0 : -1.0;
      const double wm[4] = {S.jt_kind[2 * j + s] == 1 ? 0.0 : sg, sg * v.x, sg * v.y, sg * v.z};
      for (int m = 0; m < 4; ++m) {
        node[4 * s + m] = b >= 0 ? S.nf + 4 * b + m : -1;
        w[4 * s + m] = b >= 0 ? wm[m] : 0.0;
        if (b >= 0) r = r + w[4 * s + m] * ld3(z, node[4 * s + m]);
      }
    }
    const double k = S.jt_k[j];
    e = 0.5 * k * dot(r, r);
    if (S.E_sc) scene_energy(S, S.node_scene[node[0]], 6, e);
    if (mode >= 1)
      for (int m = 0; m < 8; ++m)
        if (node[m] >= 0 && w[m] != 0.0) {
          acc_add3(g, node[m], (scale * k * w[m]) * r, S.err);
        }
    if (mode >= 2)
      for (int m = 0; m < 8; ++m)
        for (int n = 0; n < 8; ++n) {
          const double c = scale * k * w[m] * w[n];
          const int blk = S.jt_blk[64 * j + 8 * m + n];
          if (c == 0.0 || blk < 0) continue;
          acc_t* dst = Hval + 27 * (size_t)blk;
          acc_add(dst, c, S.err);
          acc_add(dst + 12, c, S.err);
          acc_add(dst + 24, c, S.err);
        }
  }
  const double s = block_sum(e);
  if (threadIdx.x == 0) acc_add(E, s, S.err);
}

// The same energy, gradient and projected Hessian with one warp per body: the
// 9x9 Hessian is built by the lanes in shared memory (padded to 10 x 10 with a
// zero row and column, which keeps eigenvalue 0) and projected by the warp's
// parallel Jacobi, so a body costs microseconds instead of a serial 9x9 sweep.
constexpr int ORTH_WARPS = 4;
struct OrthWork {
  double H[144];
  double V[144];
  double lam[12];
  double rc[6], rs[6];
  int rp[6], rq[6];
};

__global__ void __launch_bounds__(32 * ORTH_WARPS) k_abd_orth_warp(DevScene S, const double* __restrict__ z,
                                                                    double kappa_A, double scale, int mode, int project,
                                                                    acc_t* __restrict__ g, acc_t* __restrict__ Hval,
                                                                    acc_t* __restrict__ E) {
  __shared__ OrthWork work[ORTH_WARPS];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * ORTH_WARPS + wid;
  if (b >= S.nab) return;  // whole warps leave together
  OrthWork& W = work[wid];
  const int base = S.nf + 4 * b;
  const d3 a[3] = {ld3(z, base + 1), ld3(z, base + 2), ld3(z, base + 3)};
  const double k = kappa_A * S.abd_vol[b];
  double G[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G[i][j] = dot(a[i], a[j]) - (i == j ? 1.0 : 0.0);
  if (lane == 0) {
    double e = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) e += G[i][j] * G[i][j];
    acc_add(E, k * e, S.err);
    if (S.E_sc) scene_energy(S, S.node_scene[base], 5, k * e);
  }
  if (mode >= 1 && lane < 9) {
    const int i = lane / 3, c = lane % 3;
    const double gi = 4.0 * k * (G[i][0] * comp(a[0], c) + G[i][1] * comp(a[1], c) + G[i][2] * comp(a[2], c));
    acc_add(g + 3 * (3 * (base + 1 + i) + c), scale * gi, S.err);
  }
  if (mode < 2) return;
  for (int e = lane; e < 144; e += 32) {
    const int row = e / 12, col = e % 12;
    double h = 0.0;
    if (row < 9 && col < 9) {
      const int ki = row / 3, r = row % 3, li = col / 3, c = col % 3;
      h = comp(a[li], r) * comp(a[ki], c) + (r == c ? G[ki][li] : 0.0);
      if (ki == li) h += comp(a[0], r) * comp(a[0], c) + comp(a[1], r) * comp(a[1], c) + comp(a[2], r) * comp(a[2], c);
      h *= 4.0 * k;
    }
    W.H[e] = h;
  }
  __syncwarp();
  if (project) warp_project_psd(W.H, W.V, W.lam, W.rp, W.rq, W.rc, W.rs, 10, lane);
  for (int e = lane; e < 81; e += 32) {
    const int row = e / 9, col = e % 9;
    const int ki = row / 3, r = row % 3, li = col / 3, c = col % 3;
    acc_t* dst = Hval + 27 * (size_t)S.abd_blk[16 * b + 4 * (1 + ki) + (1 + li)];
    acc_add(dst + 3 * (3 * r + c), scale * W.H[12 * row + col], S.err);
  }
}

// z_out = z + alpha p ; xk_out = alpha == 1 ? xk_hat : xk + alpha pD
__global__ void k_trial(int ndof, int nk3, const double* __restrict__ z, const double* __restrict__ p, double alpha,
                        double* __restrict__ z_out, const double* __restrict__ xk, const double* __restrict__ pD,
                        const double* __restrict__ xk_hat, double* __restrict__ xk_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ndof) z_out[i] = z[i] + alpha * p[i];
  if (i < nk3) xk_out[i] = (alpha == 1.0) ? xk_hat[i] : xk[i] + alpha * pD[i];
}

__global__ void k_velocity(int ndof, const double* __restrict__ z, const double* __restrict__ z_t, double inv_dt,
                           double* __restrict__ zd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ndof) zd[i] = (z[i] - z_t[i]) * inv_dt;
}

// max |p_F| and max |p_D| into out[0], out[1] (as ordered bits of non-negative doubles)
__global__ void k_pnorm(int ndof, const double* __restrict__ p, int nk3, const double* __restrict__ pD,
                        unsigned long long* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double a = (i < ndof) ? fabs(p[i]) : 0.0;
  double b = (i < nk3) ? fabs(pD[i]) : 0.0;
  bool bad = (i < ndof && !isfinite(p[i]));
  a = block_max(bad ? 1e300 : a);
  if (threadIdx.x == 0) atomicMax(out, dbits(a));
  b = block_max(b);
  if (threadIdx.x == 0) atomicMax(out + 1, dbits(b));
}

// Batches: max |p_F| and max |p_D| per scene.
__global__ void k_pnorm_scenes(DevScene S, int ndof, const double* __restrict__ p, int nk3,
                               const double* __restrict__ pD) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ndof) {
    const double a = isfinite(p[i]) ? fabs(p[i]) : 1e300;
    if (a > 0.0) atomicMax(S.pn_sc + 2 * S.node_scene[i / 3], dbits(a));
  }
  if (i < nk3 && pD[i] != 0.0) {
    const int v = S.nf + S.na_v + i / 3;
    atomicMax(S.pn_sc + 2 * scene_of_vertex(S, v) + 1, dbits(fabs(pD[i])));
  }
}

// Batches: z_out = z + alpha_s p and xk_out = (alpha_s == 1 ? xk_hat : xk + alpha_s pD) with the step of each scene.
__global__ void k_trial_scenes(DevScene S, int ndof, int nk3, const double* __restrict__ z, const double* __restrict__ p,
                               double* __restrict__ z_out, const double* __restrict__ xk, const double* __restrict__ pD,
                               const double* __restrict__ xk_hat, double* __restrict__ xk_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ndof) z_out[i] = z[i] + S.alpha_trial[S.node_scene[i / 3]] * p[i];
  if (i < nk3) {
    const double al = S.alpha_trial[scene_of_vertex(S, S.nf + S.na_v + i / 3)];
    xk_out[i] = (al == 1.0) ? xk_hat[i] : xk[i] + al * pD[i];
  }
}

// p_D = xk_hat - xk
__global__ void k_sub(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ o) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = a[i] - b[i];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline int nb(int n, int t) { return (n + t - 1) / t; }

void launch_predict(cudaStream_t st, const DevScene& S, const double* z, const double* zd, double dt, const double* g,
                    double* z_t, double* z_tilde) {
  if (S.n_nodes) { k_predict<<<nb(S.n_nodes, 256), 256, 0, st>>>(S.n_nodes, S.nf, z, zd, dt, mk(g[0], g[1], g[2]), z_t, z_tilde); count_launch(); }
}
void launch_kin_targets(cudaStream_t st, const DevScene& S, const double* T, double* xk_hat, double* stitch_hat) {
  int n = S.nk > S.n_stitch ? S.nk : S.n_stitch;
  if (n) { k_kin_targets<<<nb(n, 256), 256, 0, st>>>(S, T, xk_hat, stitch_hat); count_launch(); }
}
void launch_vertex_positions(cudaStream_t st, const DevScene& S, const double* z, const double* xk, double* xv) {
  if (S.nv) { k_vertex_positions<<<nb(S.nv, 256), 256, 0, st>>>(S, z, xk, xv); count_launch(); }
}
void launch_vertex_disp(cudaStream_t st, const DevScene& S, const double* p, const double* pD, double* pv) {
  if (S.nv) { k_vertex_disp<<<nb(S.nv, 256), 256, 0, st>>>(S, p, pD, pv); count_launch(); }
}
void launch_inertia(cudaStream_t st, const DevScene& S, const double* z, const double* z_tilde, acc_t* g, acc_t* E,
                    int want_grad) {
  if (S.n_nodes) { k_inertia<<<nb(S.n_nodes, 256), 256, 0, st>>>(S, z, z_tilde, g, E, want_grad); count_launch(); }
}
void launch_elastic(cudaStream_t st, const DevScene& S, const double* xv, double scale, int mode, int project,
                    acc_t* g, double* tetH, acc_t* E, int hess_fp32) {
  if (!S.nt) return;
  if (hess_fp32 && mode >= 2 && project)
    k_elastic<true><<<nb(S.nt, 128), 128, 0, st>>>(S, xv, scale, mode, project, g, nullptr, nullptr, tetH, E);
  else
    k_elastic<false><<<nb(S.nt, 128), 128, 0, st>>>(S, xv, scale, mode, project, g, nullptr, nullptr, tetH, E);
  count_launch();
}

// FEM BSR blocks from the tets' stored upper triangles: Hval[k] = Hconst[k] + the 3x3 parts of the tets of
// block k, added in tet order (one thread per value; no atomics, the same order in every run)
__global__ void k_elastic_gather_H(DevScene S, const double* __restrict__ tU, const double* __restrict__ Hc,
                                   double* __restrict__ Hval) {
  const size_t n = 9 * (size_t)S.nfb;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / 9), q = (int)(i - 9 * (size_t)k), bi = q / 3, bj = q - 3 * (q / 3);
    double sum = 0.0;
    for (int l = S.eg_blk_ptr[k]; l < S.eg_blk_ptr[k + 1]; ++l) {
      const int code = S.eg_blk_ent[l], e = code >> 4, a = (code >> 2) & 3, b = code & 3;
      const int row = 3 * a + bi, col = 3 * b + bj;
      const int r = row < col ? row : col, c = row < col ? col : row;
      sum += tU[78 * (size_t)e + 12 * r - r * (r - 1) / 2 + (c - r)];
    }
    Hval[i] = Hc[i] + sum;
  }
}

// FEM node gradients from the tets' stored gradients, added in tet order, then into the accumulators
__global__ void k_elastic_gather_g(DevScene S, const double* __restrict__ tG, acc_t* __restrict__ g) {
  const int n = 3 * S.nf;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int v = i / 3, c = i - 3 * (i / 3);
    double sum = 0.0;
    for (int l = S.eg_node_ptr[v]; l < S.eg_node_ptr[v + 1]; ++l) {
      const int code = S.eg_node_ent[l];
      sum += tG[12 * (size_t)(code >> 2) + 3 * (code & 3) + c];
    }
    acc_add(g + 3 * (size_t)i, sum, S.err);
  }
}

void launch_elastic_assembly(cudaStream_t st, const DevScene& S, const double* xv, double scale, int project, acc_t* g,
                             const double* Hconst, double* Hval, acc_t* E, int hess_fp32, double* tU, double* tG) {
  if (S.nt) {
    if (hess_fp32 && project)
      k_elastic<true><<<nb(S.nt, 128), 128, 0, st>>>(S, xv, scale, 2, project, nullptr, tG, tU, nullptr, E);
    else
      k_elastic<false><<<nb(S.nt, 128), 128, 0, st>>>(S, xv, scale, 2, project, nullptr, tG, tU, nullptr, E);
    k_elastic_gather_g<<<stride_grid(3LL * S.nf, 256, 8), 256, 0, st>>>(S, tG, g);
    count_launch(2);
  }
  if (S.nfb) {  // FEM nodes without tets still take their mass and stitch blocks
    k_elastic_gather_H<<<stride_grid(9LL * S.nfb, 256, 8), 256, 0, st>>>(S, tU, Hconst, Hval);
    count_launch();
  }
}
void launch_stitch(cudaStream_t st, const DevScene& S, const double* xv, const double* stitch_hat, double k_c,
                   double scale, int mode, acc_t* g, acc_t* E) {
  if (S.n_stitch) { k_stitch<<<nb(S.n_stitch, 256), 256, 0, st>>>(S, xv, stitch_hat, k_c, scale, mode, g, E); count_launch(); }
}
void launch_abd_orth(cudaStream_t st, const DevScene& S, const double* z, double kappa_A, double scale, int mode,
                     int project, acc_t* g, acc_t* Hval, acc_t* E) {
  if (S.nab) {
    if (mode >= 2)
      k_abd_orth_warp<<<nb(S.nab, ORTH_WARPS), 32 * ORTH_WARPS, 0, st>>>(S, z, kappa_A, scale, mode, project, g, Hval, E);
    else
      k_abd_orth<<<nb(S.nab, 64), 64, 0, st>>>(S, z, kappa_A, scale, mode, project, g, Hval, E);
    count_launch();
  }
}
__global__ void k_acc_finalize(size_t n, const acc_t* __restrict__ acc, const double* __restrict__ base,
                               double* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = acc_value(acc + 3 * i);
    out[i] = base ? base[i] + v : v;
  }
}
void launch_acc_finalize(cudaStream_t st, size_t n, const acc_t* acc, const double* base, double* out) {
  if (!n) return;
  k_acc_finalize<<<stride_grid((long long)n, 256, 8), 256, 0, st>>>(n, acc, base, out);
  count_launch();
}
void launch_joints(cudaStream_t st, const DevScene& S, const double* z, double scale, int mode, acc_t* g, acc_t* Hval,
                   acc_t* E) {
  if (S.nj) { k_joints<<<nb(S.nj, 64), 64, 0, st>>>(S, z, scale, mode, g, Hval, E); count_launch(); }
}
void launch_trial(cudaStream_t st, int ndof, int nk3, const double* z, const double* p, double alpha, double* z_out,
                  const double* xk, const double* pD, const double* xk_hat, double* xk_out) {
  int n = ndof > nk3 ? ndof : nk3;
  if (n) { k_trial<<<nb(n, 256), 256, 0, st>>>(ndof, nk3, z, p, alpha, z_out, xk, pD, xk_hat, xk_out); count_launch(); }
}
void launch_velocity(cudaStream_t st, int ndof, const double* z, const double* z_t, double inv_dt, double* zd) {
  if (ndof) { k_velocity<<<nb(ndof, 256), 256, 0, st>>>(ndof, z, z_t, inv_dt, zd); count_launch(); }
}
void launch_pnorm(cudaStream_t st, int ndof, const double* p, int nk3, const double* pD, unsigned long long* out) {
  int n = ndof > nk3 ? ndof : nk3;
  if (n) { k_pnorm<<<nb(n, 256), 256, 0, st>>>(ndof, p, nk3, pD, out); count_launch(); }
}
void launch_pnorm_scenes(cudaStream_t st, const DevScene& S, int ndof, const double* p, int nk3, const double* pD) {
  int n = ndof > nk3 ? ndof : nk3;
  if (n) { k_pnorm_scenes<<<nb(n, 256), 256, 0, st>>>(S, ndof, p, nk3, pD); count_launch(); }
}
void launch_trial_scenes(cudaStream_t st, const DevScene& S, int ndof, int nk3, const double* z, const double* p,
                         double* z_out, const double* xk, const double* pD, const double* xk_hat, double* xk_out) {
  int n = ndof > nk3 ? ndof : nk3;
  if (n) {
    k_trial_scenes<<<nb(n, 256), 256, 0, st>>>(S, ndof, nk3, z, p, z_out, xk, pD, xk_hat, xk_out);
    count_launch();
  }
}
void launch_sub(cudaStream_t st, int n, const double* a, const double* b, double* o) {
  if (n) { k_sub<<<nb(n, 256), 256, 0, st>>>(n, a, b, o); count_launch(); }
}

}  // namespace ipc
