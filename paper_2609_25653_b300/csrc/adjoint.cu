// Kernels of the implicit adjoint of one step (implicit function theorem).
//
// At the converged z* the free-DOF gradient g(z*; z_t, zd_t, theta) is zero.
// With H the unprojected Hessian at z* and lam = H^-1 (dL/dz* + dL/dzd* / dt):
//   dL/dlogE_e = -dt^2 lam_e . grad(V_e Psi_e)    (Psi linear in mu, lam_m, both ~ E)
//   dL/dmu     = -dt^2 lam . grad(D) / mu
//   dL/dz_t    = M lam - dL/dzd* / dt + dt^2 H_fric lam,   dL/dzd_t = dt M lam.
#include "common.cuh"
#include "kernels.h"

namespace ipc {

// out[e] += -scale * sum_a lam_{tet_a} . grad_a(V_e Psi_e)   (scale = dt^2)
__global__ void k_theta_grad(DevScene S, const double* __restrict__ xv, const double* __restrict__ lam, double scale,
                             double* __restrict__ out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= S.nt) return;
  int4 t = S.tets[e];
  int id[4] = {t.x, t.y, t.z, t.w};
  d3 x0 = ld3(xv, id[0]);
  d3 c1 = ld3(xv, id[1]) - x0, c2 = ld3(xv, id[2]) - x0, c3 = ld3(xv, id[3]) - x0;
  const double* B = S.B + 9 * e;
  d3 f[3];
  for (int j = 0; j < 3; ++j) f[j] = B[j] * c1 + B[3 + j] * c2 + B[6 + j] * c3;
  d3 cf[3] = {cross(f[1], f[2]), cross(f[2], f[0]), cross(f[0], f[1])};
  double J = dot(f[0], cf[0]);
  double mu = S.mu[e], lm = S.lam[e], V = S.vol[e];
  double kJ = lm * (J - 1.0) - mu;
  d3 Pc[3];
  for (int j = 0; j < 3; ++j) Pc[j] = mu * f[j] + kJ * cf[j];
  double s = 0.0;
  for (int a = 0; a < 4; ++a) {
    double c[3];
    for (int j = 0; j < 3; ++j) c[j] = a == 0 ? -(B[j] + B[3 + j] + B[6 + j]) : B[3 * (a - 1) + j];
    d3 ga = c[0] * Pc[0] + c[1] * Pc[1] + c[2] * Pc[2];
    s += dot(ga, ld3(lam, id[a]));
  }
  out[e] += -scale * V * s;
}

// y = M lam over all nodes (FEM lumped masses, ABD S (x) I3); also yd = dt * y
__global__ void k_mass_apply(DevScene S, const double* __restrict__ lam, double dt, double* __restrict__ y,
                             double* __restrict__ yd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n_nodes) return;
  d3 r;
  if (i < S.nf) r = S.node_mass[i] * ld3(lam, i);
  else {
    int b = (i - S.nf) / 4, q = (i - S.nf) % 4;
    const double* Sm = S.abd_S + 16 * b;
    r = mk(0, 0, 0);
    for (int s = 0; s < 4; ++s) r = r + Sm[4 * q + s] * ld3(lam, S.nf + 4 * b + s);
  }
  st3(y, i, r);
  st3(yd, i, dt * r);
}

// y += (w w^T (x) Hu) lam for every friction pair (Hu already scaled by dt^2), into accumulators.
__global__ void k_friction_apply(DevScene S, int n, const int* __restrict__ f_ids, const double* __restrict__ f_w,
                                 const double* __restrict__ f_Hu, const double* __restrict__ lam,
                                 acc_t* __restrict__ y) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int* ids = f_ids + 4 * k;
  const double* w = f_w + 4 * k;
  const double* Hu = f_Hu + 9 * k;
  d3 U = mk(0, 0, 0);
  for (int q = 0; q < 4; ++q) {
    if (S.vkind[ids[q]] == VK_KIN || w[q] == 0.0) continue;
    NodeMap m = vertex_nodes(S, ids[q]);
    for (int t = 0; t < m.n; ++t) U = U + (w[q] * m.w[t]) * ld3(lam, m.node[t]);
  }
  d3 tv = mk(Hu[0] * U.x + Hu[1] * U.y + Hu[2] * U.z, Hu[3] * U.x + Hu[4] * U.y + Hu[5] * U.z,
             Hu[6] * U.x + Hu[7] * U.y + Hu[8] * U.z);
  for (int q = 0; q < 4; ++q) {
    if (S.vkind[ids[q]] == VK_KIN || w[q] == 0.0) continue;
    NodeMap m = vertex_nodes(S, ids[q]);
    for (int t = 0; t < m.n; ++t) {
      acc_add3(y, m.node[t], (w[q] * m.w[t]) * tv, S.err);
    }
  }
}

// out (accumulator) += sum_i a_i b_i
__global__ void k_dot(int n, const double* __restrict__ a, const double* __restrict__ b, acc_t* __restrict__ out) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += a[i] * b[i];
  s = block_sum(s);
  if (threadIdx.x == 0) acc_add(out, s);
}

// a = gz + gzd / dt (free DOFs); also used for gz_t -= gzd / dt
__global__ void k_axpy(int n, const double* __restrict__ x, double alpha, const double* __restrict__ y,
                       double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = x[i] + alpha * y[i];
}

static int nb(int n, int t) { return (n + t - 1) / t; }

void launch_theta_grad(cudaStream_t st, const DevScene& S, const double* xv, const double* lam, double scale, double* out) {
  if (S.nt) { k_theta_grad<<<nb(S.nt, 128), 128, 0, st>>>(S, xv, lam, scale, out); count_launch(); }
}
void launch_mass_apply(cudaStream_t st, const DevScene& S, const double* lam, double dt, double* y, double* yd) {
  if (S.n_nodes) { k_mass_apply<<<nb(S.n_nodes, 256), 256, 0, st>>>(S, lam, dt, y, yd); count_launch(); }
}
void launch_friction_apply(cudaStream_t st, const DevScene& S, int n, const int* f_ids, const double* f_w,
                           const double* f_Hu, const double* lam, acc_t* y) {
  if (n > 0) { k_friction_apply<<<nb(n, 128), 128, 0, st>>>(S, n, f_ids, f_w, f_Hu, lam, y); count_launch(); }
}
void launch_dot(cudaStream_t st, int n, const double* a, const double* b, acc_t* out) {
  if (n > 0) { k_dot<<<stride_grid(n, 256, 4), 256, 0, st>>>(n, a, b, out); count_launch(); }
}
void launch_axpy(cudaStream_t st, int n, const double* x, double alpha, const double* y, double* out) {
  if (n > 0) { k_axpy<<<nb(n, 256), 256, 0, st>>>(n, x, alpha, y, out); count_launch(); }
}

}  // namespace ipc
