// Contact kernels: log-barrier energy, gradient and PSD-projected Hessian per
// point-triangle / edge-edge pair (E_barrier of Eq. 3), the edge-edge
// mollifier, lagged friction (E_friction of Eq. 3), and the Dirichlet
// coupling of kinematic vertices.
//
// Barrier (on squared distance s, sh = dhat^2): b(s) = -(s - sh)^2 ln(s / sh)
// for 0 < s < sh.  Pair energy kappa * m * b(s), m the edge-edge mollifier
// (1 for point-triangle pairs).  Friction per lagged pair: mu * lambda *
// f0(|P u|), u = sum_k w_k (x_k - x_t,k), P = I - n n^T, f0 the C1 cubic
// below eps = eps_v dt.
#include "common.cuh"
#include "dist.cuh"
#include "eig.cuh"
#include "kernels.h"
#include <algorithm>

namespace ipc {

__device__ inline void barrier_fn(double s, double sh, double& b, double& b1, double& b2) {
  if (s >= sh) { b = b1 = b2 = 0.0; return; }
  double d = s - sh, l = log(s / sh);
  b = -d * d * l;
  b1 = -(2.0 * d * l + d * d / s);
  b2 = -(2.0 * l + 4.0 * d / s - d * d / (s * s));
}

// Edge-edge mollifier value m(c) = -(c/eps)^2 + 2 c/eps below eps, else 1; c = |(a1-a0) x (b1-b0)|^2.
__device__ inline double moll_value(const d3* x, double eps_x) {
  d3 n = cross(x[1] - x[0], x[3] - x[2]);
  double c = dot(n, n);
  if (c >= eps_x) return 1.0;
  double r = c / eps_x;
  return -r * r + 2.0 * r;
}

// Edge-edge mollifier m(c): value, gradient g and Hessian H (c < eps_x assumed by callers that use g/H).
__device__ inline double mollifier(const d3* x, double eps_x, double* g, double* H) {
  d3 a = x[1] - x[0], b = x[3] - x[2];
  d3 n = cross(a, b);
  double c = dot(n, n);
  if (c >= eps_x) return 1.0;
  double r = c / eps_x;
  double m = -r * r + 2.0 * r;
  double m1 = (2.0 - 2.0 * r) / eps_x, m2 = -2.0 / (eps_x * eps_x);
  d3 ga = 2.0 * cross(b, n), gb = 2.0 * cross(n, a);
  double gc[12] = {-ga.x, -ga.y, -ga.z, ga.x, ga.y, ga.z, -gb.x, -gb.y, -gb.z, gb.x, gb.y, gb.z};
  for (int i = 0; i < 12; ++i) g[i] = m1 * gc[i];
  if (!H) return m;
  double Sa[9], Sb[9], Sn[9], Haa[9], Hbb[9], Hab[9], T[9];
  skew9(a, Sa);
  skew9(b, Sb);
  skew9(n, Sn);
  mm3(Sb, Sb, T);
  for (int i = 0; i < 9; ++i) Haa[i] = -2.0 * T[i];
  mm3(Sa, Sa, T);
  for (int i = 0; i < 9; ++i) Hbb[i] = -2.0 * T[i];
  mm3(Sb, Sa, T);
  for (int i = 0; i < 9; ++i) Hab[i] = 2.0 * T[i] - 2.0 * Sn[i];
  // slot coefficients: a = x1 - x0, b = x3 - x2
  const double ca[4] = {-1, 1, 0, 0}, cb[4] = {0, 0, -1, 1};
  for (int k = 0; k < 4; ++k)
    for (int l = 0; l < 4; ++l)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double h = ca[k] * ca[l] * Haa[3 * i + j] + cb[k] * cb[l] * Hbb[3 * i + j] + ca[k] * cb[l] * Hab[3 * i + j] +
                     cb[k] * ca[l] * Hab[3 * j + i];
          H[12 * (3 * k + i) + 3 * l + j] = m2 * gc[3 * k + i] * gc[3 * l + j] + m1 * h;
        }
  return m;
}

__device__ inline void load_stencil(const DevScene& S, const double* xv, const int* r, int* ids, d3* x) {
  for (int k = 0; k < 4; ++k) {
    ids[k] = r[4 + k];
    x[k] = ld3(xv, ids[k]);
  }
}

// slots of the stencil that the distance of (kind, type) depends on
__device__ inline int involved_mask(int kind, int type) {
  if (kind == 0) {
    if (type <= 2) return 1 | (2 << type);
    if (type <= 5) return 1 | (2 << (type - 3)) | (2 << ((type - 2) % 3));
    return 15;
  }
  if (type <= 3) return (1 << (type / 2)) | (4 << (type % 2));
  if (type <= 5) return 3 | (4 << (type - 4));
  if (type <= 7) return 12 | (1 << (type - 6));
  return 15;
}

// Project the sub-block of the slots in `mask` (other rows/columns are zero).
__device__ inline void project_pair(double* H, int mask) {
  int sl[4], ns = 0;
  for (int k = 0; k < 4; ++k)
    if (mask & (1 << k)) sl[ns++] = k;
  if (ns == 4) { project_psd<12, double>(H); return; }
  double A[81];
  int n = 3 * ns;
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[n * (3 * a + i) + 3 * b + j] = H[12 * (3 * sl[a] + i) + 3 * sl[b] + j];
  if (ns == 2) project_psd<6, double>(A);
  else project_psd<9, double>(A);
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[12 * (3 * sl[a] + i) + 3 * sl[b] + j] = A[n * (3 * a + i) + 3 * b + j];
}

// Scatter a vertex-space 12-vector (scaled) to node space.
__device__ inline void scatter_grad(const DevScene& S, const int* ids, const double* gv, double scale, acc_t* g) {
  for (int k = 0; k < 4; ++k) {
    NodeMap m = vertex_nodes(S, ids[k]);
    for (int r = 0; r < m.n; ++r) {
      double w = scale * m.w[r];
      acc_add(g + 3 * ((size_t)(3 * m.node[r])), w * gv[3 * k], S.err);
      acc_add(g + 3 * ((size_t)(3 * m.node[r] + 1)), w * gv[3 * k + 1], S.err);
      acc_add(g + 3 * ((size_t)(3 * m.node[r] + 2)), w * gv[3 * k + 2], S.err);
    }
  }
}

// Diagonal node blocks of J^T H J (for the block-Jacobi preconditioner) and
// H_FD p_D (the Dirichlet coupling) of a dense 12x12 vertex-space block.
__device__ inline void scatter_diag_dirichlet(const DevScene& S, const int* ids, const double* H, const double* pD,
                                              acc_t* Dc, acc_t* gdir) {
  NodeMap m[4];
  bool kin[4];
  d3 pk[4];
  for (int k = 0; k < 4; ++k) {
    m[k] = vertex_nodes(S, ids[k]);
    kin[k] = S.vkind[ids[k]] == VK_KIN;
    pk[k] = kin[k] ? ld3(pD, ids[k] - S.nf - S.na_v) : mk(0, 0, 0);
  }
  for (int a = 0; a < 4; ++a) {
    if (kin[a]) continue;
    // Dirichlet: y_a = sum_{kinematic b} H_ab pD_b
    d3 y = mk(0, 0, 0);
    for (int b = 0; b < 4; ++b) {
      if (!kin[b]) continue;
      const double* Hr = H + 12 * 3 * a + 3 * b;
      y = y + mk(Hr[0] * pk[b].x + Hr[1] * pk[b].y + Hr[2] * pk[b].z, Hr[12] * pk[b].x + Hr[13] * pk[b].y + Hr[14] * pk[b].z,
                 Hr[24] * pk[b].x + Hr[25] * pk[b].y + Hr[26] * pk[b].z);
    }
    if (y.x != 0.0 || y.y != 0.0 || y.z != 0.0)
      for (int r = 0; r < m[a].n; ++r) {
        acc_add(gdir + 3 * ((size_t)(3 * m[a].node[r])), m[a].w[r] * y.x, S.err);
        acc_add(gdir + 3 * ((size_t)(3 * m[a].node[r] + 1)), m[a].w[r] * y.y, S.err);
        acc_add(gdir + 3 * ((size_t)(3 * m[a].node[r] + 2)), m[a].w[r] * y.z, S.err);
      }
    // diagonal node blocks
    for (int b = 0; b < 4; ++b) {
      if (kin[b]) continue;
      for (int r = 0; r < m[a].n; ++r)
        for (int q = 0; q < m[b].n; ++q) {
          if (m[a].node[r] != m[b].node[q]) continue;
          double w = m[a].w[r] * m[b].w[q];
          acc_t* dst = Dc + 27 * (size_t)m[a].node[r];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) acc_add(dst + 3 * (3 * i + j), w * H[12 * (3 * a + i) + 3 * b + j], S.err);
        }
    }
  }
}

// mode 0: energy (and min s) only; mode 2: also gradient, projected Hessian, preconditioner diagonal, Dirichlet term.
__global__ void __launch_bounds__(128) k_barrier(DevScene S, const double* __restrict__ xv, const int* __restrict__ rec,
                                                 const int* __restrict__ n_dev, int cap, double sh, double kappa_unused,
                                                 double scale, int mode, int project, acc_t* __restrict__ g,
                                                 double* __restrict__ pairH, acc_t* __restrict__ Dc,
                                                 const double* __restrict__ pD, acc_t* __restrict__ gdir,
                                                 acc_t* __restrict__ E, unsigned long long* __restrict__ min_s) {
  int n = min(*n_dev, cap);
  double smin = 1e300;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    {
      const int* r = rec + 8 * (size_t)k;
      int kind = r[0], type = r[3];
      int ids[4];
      d3 x[4];
      load_stencil(S, xv, r, ids, x);
      const double kappa = S.scene_kappa[scene_of_vertex(S, ids[0])];
      Red R;
      double s;
      dist_reduced(kind, type, x, R, s);
      smin = fmin(smin, s);
      double b, b1, b2;
      barrier_fn(s, sh, b, b1, b2);
      double eps_x = kind == 1 ? 1e-3 * S.edge_rest_sq[r[1]] * S.edge_rest_sq[r[2]] : 0.0;
      if (mode == 0) {
        double m = kind == 1 ? moll_value(x, eps_x) : 1.0;
        acc_add(S.e_slots + 3 * (k & (E_SLOTS - 1)), kappa * m * b, S.err);
        if (S.E_sc) scene_energy(S, scene_of_vertex(S, ids[0]), 2, kappa * m * b);
      } else if (b != 0.0 || b1 != 0.0) {
        double gs[12], Hs[144];
        red_expand(R, gs, Hs);
        double gm[12], Hm[144];
        double m = 1.0;
        bool moll = false;
        if (kind == 1) {
          d3 a = x[1] - x[0], bb = x[3] - x[2];
          d3 nn = cross(a, bb);
          if (dot(nn, nn) < eps_x) { m = mollifier(x, eps_x, gm, Hm); moll = true; }
        }
        acc_add(S.e_slots + 3 * (k & (E_SLOTS - 1)), kappa * m * b, S.err);
        if (S.E_sc) scene_energy(S, scene_of_vertex(S, ids[0]), 2, kappa * m * b);
        double grad[12];
        for (int i = 0; i < 12; ++i) grad[i] = kappa * (m * b1 * gs[i] + (moll ? b * gm[i] : 0.0));
        double* H = pairH + 144 * (size_t)k;
        for (int i = 0; i < 12; ++i)
          for (int j = 0; j < 12; ++j) {
            double h = m * (b2 * gs[i] * gs[j] + b1 * Hs[12 * i + j]);
            if (moll) h += b * Hm[12 * i + j] + b1 * (gm[i] * gs[j] + gs[i] * gm[j]);
            Hs[12 * i + j] = kappa * h;
          }
        if (project) project_pair(Hs, moll ? 15 : involved_mask(kind, type));
        for (int i = 0; i < 144; ++i) {
          Hs[i] *= scale;
          H[i] = Hs[i];
        }
        scatter_grad(S, ids, grad, scale, g);
        scatter_diag_dirichlet(S, ids, Hs, pD, Dc, gdir);
      } else {
        double* H = pairH + 144 * (size_t)k;
        for (int i = 0; i < 144; ++i) H[i] = 0.0;
      }
    }
  }
  double m = block_max(-smin);
  if (threadIdx.x == 0 && min_s) atomicMin(min_s, dbits(-m));
}


// ---------------------------------------------------------------------------
// warp-cooperative barrier assembly: one warp per pair
// ---------------------------------------------------------------------------
// Lane 0 evaluates the reduced distance derivatives, the barrier scalars and
// the mollifier pieces; the 12x12 Hessian entries, its PSD projection
// (parallel cyclic Jacobi: n/2 disjoint rotations per round, round-robin
// pairing, n - 1 rounds per sweep) and every scatter are spread over the
// lanes, with the matrices in shared memory.
constexpr int BWARPS = 4;

struct PairWork {
  double H[144];
  double V[144];
  double RH[81];
  double Rg[9];
  double C[12];
  double gs[12];
  double gc[12];
  double mH[27];   // mollifier pieces: Haa, Hbb, Hab (3x3 each)
  double sc[8];    // s, b, b1, b2, m, m1, m2
  double rc[6], rs[6];
  double lam[12];
  int rp[6], rq[6];
  int idx[12];
  int ids[4];
  int nvar, moll, n;
};

// PSD projection of W.H (n x n, n even <= 12, row stride 12) in place (eig.cuh)
__device__ inline void warp_project(PairWork& W, int n, int lane) {
  warp_project_psd<double>(W.H, W.V, W.lam, W.rp, W.rq, W.rc, W.rs, n, lane);
}
// The same projection in FP32 (mixed precision, where the solve stores the pair blocks in FP32): the
// diagonal-dominance test on the FP64 matrix, then the rotations in FP32 in the storage of W.V (free until
// the scatter), widened back into W.H.  The barrier value, its derivatives and the gradient stay FP64.
__device__ inline void warp_project_f32(PairWork& W, int n, int lane) {
  bool dom = true;
  if (lane < n) {
    double off = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != lane) off += fabs(W.H[12 * lane + j]);
    dom = W.H[13 * lane] >= off;
  }
  if (__all_sync(0xffffffffu, dom)) return;
  float* A = reinterpret_cast<float*>(W.V);
  float* V = A + 144;
  for (int e = lane; e < 144; e += 32) A[e] = (float)W.H[e];
  __syncwarp();
  warp_project_psd<float>(A, V, reinterpret_cast<float*>(W.lam), W.rp, W.rq, reinterpret_cast<float*>(W.rc),
                          reinterpret_cast<float*>(W.rs), n, lane);
  for (int e = lane; e < 144; e += 32) W.H[e] = (double)A[e];
  __syncwarp();
}

__global__ void __launch_bounds__(32 * BWARPS) k_barrier_warp(DevScene S, const double* __restrict__ xv,
                                                             const int* __restrict__ rec, const int* __restrict__ n_dev,
                                                             int cap, double sh, double kappa_unused, double scale,
                                                             int project, acc_t* __restrict__ g,
                                                             double* __restrict__ pairH, acc_t* __restrict__ Dc,
                                                             const double* __restrict__ pD, acc_t* __restrict__ gdir,
                                                             acc_t* __restrict__ E, unsigned long long* min_s,
                                                             int hess_fp32) {
  __shared__ PairWork work[BWARPS];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  PairWork& W = work[wid];
  int n = min(*n_dev, cap);
  double smin = 1e300;
  int gw = blockIdx.x * BWARPS + wid, nw = gridDim.x * BWARPS;
  for (int k = gw; k < n; k += nw) {
    const int* r = rec + 8 * (size_t)k;
    int kind = r[0], type = r[3];
    const double kappa = S.scene_kappa[scene_of_vertex(S, r[4])];
    if (lane == 0) {
      d3 x[4];
      for (int q = 0; q < 4; ++q) { W.ids[q] = r[4 + q]; x[q] = ld3(xv, W.ids[q]); }
      Red R;
      double sd;
      dist_reduced(kind, type, x, R, sd);
      double b, b1, b2;
      barrier_fn(sd, sh, b, b1, b2);
      W.nvar = R.nv;
      for (int m = 0; m < 3; ++m)
        for (int q = 0; q < 4; ++q) W.C[4 * m + q] = m < R.nv ? R.C[m][q] : 0.0;
      for (int m = 0; m < R.nv; ++m) { W.Rg[3 * m] = R.g[m].x; W.Rg[3 * m + 1] = R.g[m].y; W.Rg[3 * m + 2] = R.g[m].z; }
      for (int m = 0; m < R.nv; ++m)
        for (int nn = 0; nn < R.nv; ++nn)
          for (int q = 0; q < 9; ++q) W.RH[27 * m + 9 * nn + q] = R.H[m][nn][q];
      double mval = 1.0, m1 = 0.0, m2 = 0.0;
      int moll = 0;
      if (kind == 1) {
        double eps_x = 1e-3 * S.edge_rest_sq[r[1]] * S.edge_rest_sq[r[2]];
        d3 a = x[1] - x[0], bb = x[3] - x[2];
        d3 nn = cross(a, bb);
        double c = dot(nn, nn);
        if (c < eps_x) {
          moll = 1;
          double rr = c / eps_x;
          mval = -rr * rr + 2.0 * rr;
          m1 = (2.0 - 2.0 * rr) / eps_x;
          m2 = -2.0 / (eps_x * eps_x);
          d3 ga = 2.0 * cross(bb, nn), gb = 2.0 * cross(nn, a);
          double gc[12] = {-ga.x, -ga.y, -ga.z, ga.x, ga.y, ga.z, -gb.x, -gb.y, -gb.z, gb.x, gb.y, gb.z};
          for (int i = 0; i < 12; ++i) W.gc[i] = gc[i];
          double Sa[9], Sb[9], Sn[9], T[9];
          skew9(a, Sa); skew9(bb, Sb); skew9(nn, Sn);
          mm3(Sb, Sb, T);
          for (int i = 0; i < 9; ++i) W.mH[i] = -2.0 * T[i];
          mm3(Sa, Sa, T);
          for (int i = 0; i < 9; ++i) W.mH[9 + i] = -2.0 * T[i];
          mm3(Sb, Sa, T);
          for (int i = 0; i < 9; ++i) W.mH[18 + i] = 2.0 * T[i] - 2.0 * Sn[i];
        }
      }
      W.moll = moll;
      W.sc[0] = sd; W.sc[1] = b; W.sc[2] = b1; W.sc[3] = b2; W.sc[4] = mval; W.sc[5] = m1; W.sc[6] = m2;
      smin = fmin(smin, sd);
      acc_add(S.e_slots + 3 * (k & (E_SLOTS - 1)), kappa * mval * b, S.err);
      if (S.E_sc) scene_energy(S, scene_of_vertex(S, W.ids[0]), 2, kappa * mval * b);
      if (S.min_sc) atomicMin(S.min_sc + scene_of_vertex(S, W.ids[0]), dbits(sd));
    }
    __syncwarp();
    double b = W.sc[1], b1 = W.sc[2], b2 = W.sc[3], mval = W.sc[4], m1 = W.sc[5], m2 = W.sc[6];
    int nvar = W.nvar, moll = W.moll;
    double* Hout = pairH + 144 * (size_t)k;
    if (b == 0.0 && b1 == 0.0) {
      for (int e = lane; e < 144; e += 32) Hout[e] = 0.0;
      __syncwarp();
      continue;
    }
    // gradient of s (12 entries)
    if (lane < 12) {
      int q = lane / 3, d = lane % 3;
      double acc = 0.0;
      for (int m = 0; m < nvar; ++m) acc += W.C[4 * m + q] * W.Rg[3 * m + d];
      W.gs[lane] = acc;
    }
    __syncwarp();
    // Hessian entries
    for (int e = lane; e < 144; e += 32) {
      int i = e / 12, j = e % 12;
      int ka = i / 3, ii = i % 3, la = j / 3, jj = j % 3;
      double hs = 0.0;
      for (int m = 0; m < nvar; ++m) {
        double cm = W.C[4 * m + ka];
        if (cm == 0.0) continue;
        for (int nn = 0; nn < nvar; ++nn) {
          double cn = W.C[4 * nn + la];
          if (cn != 0.0) hs += cm * cn * W.RH[27 * m + 9 * nn + 3 * ii + jj];
        }
      }
      double h = mval * (b2 * W.gs[i] * W.gs[j] + b1 * hs);
      if (moll) {
        const double ca[4] = {-1, 1, 0, 0}, cb[4] = {0, 0, -1, 1};
        double hc = ca[ka] * ca[la] * W.mH[3 * ii + jj] + cb[ka] * cb[la] * W.mH[9 + 3 * ii + jj] +
                    ca[ka] * cb[la] * W.mH[18 + 3 * ii + jj] + cb[ka] * ca[la] * W.mH[18 + 3 * jj + ii];
        double hm = m2 * W.gc[i] * W.gc[j] + m1 * hc;
        double gmi = m1 * W.gc[i], gmj = m1 * W.gc[j];
        h += b * hm + b1 * (gmi * W.gs[j] + W.gs[i] * gmj);
      }
      W.V[e] = kappa * h;  // staging: full 12x12 in V
    }
    __syncwarp();
    if (project) {
      // compact the involved DOFs (padded to an even count) into H, project, scatter back
      int mask = moll ? 15 : involved_mask(kind, type);
      if (lane == 0) {
        int c = 0;
        for (int q = 0; q < 4; ++q)
          if (mask & (1 << q))
            for (int d = 0; d < 3; ++d) W.idx[c++] = 3 * q + d;
        W.n = c + (c & 1);
        if (c & 1) W.idx[c] = -1;
      }
      __syncwarp();
      int nn = W.n;
      for (int e = lane; e < 144; e += 32) {
        int a = e / 12, bcol = e % 12;
        double v = 0.0;
        if (a < nn && bcol < nn && W.idx[a] >= 0 && W.idx[bcol] >= 0) v = W.V[12 * W.idx[a] + W.idx[bcol]];
        W.H[e] = v;
      }
      __syncwarp();
      if (hess_fp32) warp_project_f32(W, nn, lane);
      else warp_project(W, nn, lane);
      // scatter H (compact) into a zeroed 12x12 in V
      for (int e = lane; e < 144; e += 32) W.V[e] = 0.0;
      __syncwarp();
      for (int e = lane; e < 144; e += 32) {
        int a = e / 12, bcol = e % 12;
        if (a < nn && bcol < nn && W.idx[a] >= 0 && W.idx[bcol] >= 0) W.V[12 * W.idx[a] + W.idx[bcol]] = W.H[e];
      }
      __syncwarp();
    }
    // scale and store
    for (int e = lane; e < 144; e += 32) {
      double v = scale * W.V[e];
      W.V[e] = v;
      Hout[e] = v;
    }
    __syncwarp();
    // gradient scatter
    if (lane < 12) {
      double gi = kappa * (mval * b1 * W.gs[lane] + (moll ? b * m1 * W.gc[lane] : 0.0));
      NodeMap m = vertex_nodes(S, W.ids[lane / 3]);
      for (int t = 0; t < m.n; ++t) acc_add(g + 3 * ((size_t)(3 * m.node[t] + lane % 3)), scale * m.w[t] * gi, S.err);
    }
    // diagonal node blocks (a, b) entry (i, j): item = (a, b, i, j), 144 items
    for (int e = lane; e < 144; e += 32) {
      int row = e / 12, col = e % 12;
      int a = row / 3, i = row % 3, bb = col / 3, j = col % 3;
      int va = W.ids[a], vb = W.ids[bb];
      if (S.vkind[va] == VK_KIN || S.vkind[vb] == VK_KIN) continue;
      NodeMap ma = vertex_nodes(S, va), mb = vertex_nodes(S, vb);
      double h = W.V[e];
      for (int t = 0; t < ma.n; ++t)
        for (int u = 0; u < mb.n; ++u)
          if (ma.node[t] == mb.node[u]) acc_add(Dc + 3 * (9 * (size_t)ma.node[t] + 3 * i + j), ma.w[t] * mb.w[u] * h, S.err);
    }
    // Dirichlet: free slot a row i: sum over kinematic slots b of H_ab pD_b
    if (lane < 12) {
      int a = lane / 3, i = lane % 3;
      int va = W.ids[a];
      if (S.vkind[va] != VK_KIN) {
        double y = 0.0;
        for (int bb = 0; bb < 4; ++bb) {
          int vb = W.ids[bb];
          if (S.vkind[vb] != VK_KIN) continue;
          d3 pk = ld3(pD, vb - S.nf - S.na_v);
          const double* Hr = W.V + 12 * (3 * a + i) + 3 * bb;
          y += Hr[0] * pk.x + Hr[1] * pk.y + Hr[2] * pk.z;
        }
        if (y != 0.0) {
          NodeMap m = vertex_nodes(S, va);
          for (int t = 0; t < m.n; ++t) acc_add(gdir + 3 * ((size_t)(3 * m.node[t] + i)), m.w[t] * y, S.err);
        }
      }
    }
    __syncwarp();
  }
  double mm = block_max(-smin);
  if (threadIdx.x == 0 && min_s) atomicMin(min_s, dbits(-mm));
}

// Lagged friction data at the start of the step for every active pair:
// closest-point weights w, unit normal n, normal force lambda = -kappa m 2 d b'(s).
__global__ void k_friction_lag(DevScene S, const double* __restrict__ xv, const int* __restrict__ rec,
                               const int* __restrict__ n_dev, int cap, double sh, double kappa_unused, int* __restrict__ f_ids,
                               double* __restrict__ f_w, double* __restrict__ f_n, double* __restrict__ f_lam,
                               int* __restrict__ f_rec) {
  int n = min(*n_dev, cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int* r = rec + 8 * (size_t)k;
    int kind = r[0];
    int ids[4];
    d3 x[4];
    load_stencil(S, xv, r, ids, x);
    double s, w[4];
    const int type = kind == 0 ? pt_classify(x, s, w) : ee_classify(x, s, w);
    if (f_rec) { f_rec[4 * k] = kind; f_rec[4 * k + 1] = type; f_rec[4 * k + 2] = r[1]; f_rec[4 * k + 3] = r[2]; }
    const double kappa = S.scene_kappa[scene_of_vertex(S, ids[0])];
    double d = sqrt(s);
    d3 nrm = (1.0 / d) * (w[0] * x[0] + w[1] * x[1] + w[2] * x[2] + w[3] * x[3]);
    double b, b1, b2;
    barrier_fn(s, sh, b, b1, b2);
    double m = kind == 1 ? moll_value(x, 1e-3 * S.edge_rest_sq[r[1]] * S.edge_rest_sq[r[2]]) : 1.0;
    for (int q = 0; q < 4; ++q) { f_ids[4 * k + q] = ids[q]; f_w[4 * k + q] = w[q]; }
    f_n[3 * k] = nrm.x; f_n[3 * k + 1] = nrm.y; f_n[3 * k + 2] = nrm.z;
    f_lam[k] = -kappa * m * 2.0 * d * b1;
  }
}

// Directions (4 slots x k) along which the closest-point weights of a
// distance type move, w = w0 + B theta (theta: the segment or barycentric
// coordinates the type leaves free); returns k (0 for point-point).
__device__ inline int weight_directions(int kind, int type, double B[4][2]) {
  for (int q = 0; q < 4; ++q) B[q][0] = B[q][1] = 0.0;
  if (kind == 0) {
    if (type <= 2) return 0;
    if (type <= 5) {
      const int k = type - 3;
      B[1 + k][0] = 1.0;
      B[1 + (k + 1) % 3][0] = -1.0;
      return 1;
    }
    B[1][0] = 1.0; B[2][0] = -1.0; B[1][1] = 1.0; B[3][1] = -1.0;
    return 2;
  }
  if (type <= 3) return 0;
  if (type <= 5) { B[0][0] = -1.0; B[1][0] = 1.0; return 1; }
  if (type <= 7) { B[2][0] = 1.0; B[3][0] = -1.0; return 1; }
  B[0][0] = -1.0; B[1][0] = 1.0; B[2][1] = 1.0; B[3][1] = -1.0;
  return 2;
}

// The part of the adjoint dL/dx_t that flows through the lagged friction data
// of every friction pair (normal force lambda, normal n and closest-point
// weights w, all computed at x_t).  For the adjoint lam (DOF space) of one
// step, per pair (v_q the vertex-space adjoint of slot q):
//   Phi = mu lambda phi(r) a.y,  a = sum_q w_q v_q,  y = (I - n n^T) u,
//   u = sum_q w_q (x_q - xt_q),  r = |y|,  phi(r) = f0'(r) / r,
// and -scale dPhi/dx_t through lambda, n and w is added into gz (DOF space;
// kinematic vertices dropped).  Within one distance type the weights
// minimise |V w|^2 over w = w0 + B theta, so with A = V B and A^T v = 0,
// dtheta = -(A^T A)^-1 (dA^T v + A^T dV w); lambda = -kappa m 2 d b'(s)
// through the squared distance s and the edge-edge mollifier m.
__global__ void k_friction_lag_adjoint(DevScene S, const double* __restrict__ xv, const double* __restrict__ xv_t,
                                       int n, const int* __restrict__ f_ids, const int* __restrict__ f_rec, double sh,
                                       double mu, double eps, double scale, const double* __restrict__ lam_dof,
                                       acc_t* __restrict__ gz) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int kind = f_rec[4 * k], ta = f_rec[4 * k + 2], tb = f_rec[4 * k + 3];
  int ids[4];
  d3 x[4], xs[4], vq[4];
  for (int q = 0; q < 4; ++q) {
    ids[q] = f_ids[4 * k + q];
    x[q] = ld3(xv_t, ids[q]);
    xs[q] = ld3(xv, ids[q]);
    const NodeMap m = vertex_nodes(S, ids[q]);
    d3 a = mk(0, 0, 0);
    for (int r = 0; r < m.n; ++r) a = a + m.w[r] * ld3(lam_dof, m.node[r]);
    vq[q] = a;
  }
  double s, w[4];
  const int type = kind == 0 ? pt_classify(x, s, w) : ee_classify(x, s, w);
  // gradient of the squared distance of this type at x_t
  double gs[12];
  {
    Red R;
    double s2;
    dist_reduced(kind, type, x, R, s2);
    red_expand(R, gs, nullptr);
  }
  const double d = sqrt(s);
  const d3 v = w[0] * x[0] + w[1] * x[1] + w[2] * x[2] + w[3] * x[3];
  const d3 nrm = (1.0 / d) * v;
  double b, b1, b2;
  barrier_fn(s, sh, b, b1, b2);
  double m = 1.0, gm[12];
  for (int i = 0; i < 12; ++i) gm[i] = 0.0;
  if (kind == 1) m = mollifier(x, 1e-3 * S.edge_rest_sq[ta] * S.edge_rest_sq[tb], gm, nullptr);
  const double kappa = S.scene_kappa[scene_of_vertex(S, ids[0])];
  const double lam = -kappa * m * 2.0 * d * b1;
  // friction state at x*
  d3 u = mk(0, 0, 0), Delta[4];
  for (int q = 0; q < 4; ++q) {
    Delta[q] = xs[q] - x[q];
    u = u + w[q] * Delta[q];
  }
  const d3 y = u - dot(nrm, u) * nrm;
  const double r = sqrt(dot(y, y));
  const double phi = r < eps ? (-r / (eps * eps) + 2.0 / eps) : 1.0 / r;
  const double dphi_r = r < eps ? (r > 0.0 ? (-1.0 / (eps * eps)) / r : 0.0) : -1.0 / (r * r * r);
  const d3 a = w[0] * vq[0] + w[1] * vq[1] + w[2] * vq[2] + w[3] * vq[3];
  const double ay = dot(a, y);
  const double c2 = mu * lam * phi, c1 = mu * lam * dphi_r * ay;
  const double phi_over_lam = mu * phi * ay;  // Phi / lambda
  const d3 zc = c1 * y + c2 * a;
  const d3 Ta = a - dot(nrm, a) * nrm;
  const d3 g_u = c1 * y + c2 * Ta;
  const double nu = dot(nrm, u), nz = dot(nrm, zc);
  const d3 g_n = -1.0 * (nu * zc + nz * u);
  double dPhi_dw[4];
  for (int q = 0; q < 4; ++q) dPhi_dw[q] = c2 * dot(y, vq[q]) + dot(g_u, Delta[q]);
  // weight derivatives: dw[q][col] for the 12 position components of x_t
  double Bm[4][2];
  const int nf = weight_directions(kind, type, Bm);
  double A[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  for (int c = 0; c < nf; ++c) {
    d3 acol = Bm[0][c] * x[0] + Bm[1][c] * x[1] + Bm[2][c] * x[2] + Bm[3][c] * x[3];
    A[0][c] = acol.x; A[1][c] = acol.y; A[2][c] = acol.z;
  }
  double Gi[2][2] = {{0, 0}, {0, 0}};
  if (nf == 1) {
    Gi[0][0] = 1.0 / (A[0][0] * A[0][0] + A[1][0] * A[1][0] + A[2][0] * A[2][0]);
  } else if (nf == 2) {
    const double g00 = A[0][0] * A[0][0] + A[1][0] * A[1][0] + A[2][0] * A[2][0];
    const double g01 = A[0][0] * A[0][1] + A[1][0] * A[1][1] + A[2][0] * A[2][1];
    const double g11 = A[0][1] * A[0][1] + A[1][1] * A[1][1] + A[2][1] * A[2][1];
    const double det = g00 * g11 - g01 * g01;
    Gi[0][0] = g11 / det; Gi[0][1] = -g01 / det; Gi[1][0] = -g01 / det; Gi[1][1] = g00 / det;
  }
  const double vv[3] = {v.x, v.y, v.z};
  double grad[12];
  for (int j = 0; j < 4; ++j)
    for (int dd = 0; dd < 3; ++dd) {
      const int col = 3 * j + dd;
      // dw[:, col] = B dtheta, dtheta = -(A^T A)^-1 (B_j v_dd + A_dd w_j)
      double dw[4] = {0, 0, 0, 0};
      if (nf) {
        double rhs[2] = {0, 0}, dth[2] = {0, 0};
        for (int c = 0; c < nf; ++c) rhs[c] = Bm[j][c] * vv[dd] + A[dd][c] * w[j];
        for (int c = 0; c < nf; ++c) dth[c] = -(Gi[c][0] * rhs[0] + Gi[c][1] * rhs[1]);
        for (int q = 0; q < 4; ++q) dw[q] = Bm[q][0] * dth[0] + Bm[q][1] * dth[1];
      }
      // dv[:, col] = e_dd w_j + sum_q x_q dw_q;  dn = (I - n n^T) dv / d
      d3 dv = dw[0] * x[0] + dw[1] * x[1] + dw[2] * x[2] + dw[3] * x[3];
      if (dd == 0) dv.x += w[j]; else if (dd == 1) dv.y += w[j]; else dv.z += w[j];
      const d3 dn = (1.0 / d) * (dv - dot(nrm, dv) * nrm);
      const double dlam = -kappa * (2.0 * d * b1 * gm[col] + m * (b1 / d + 2.0 * d * b2) * gs[col]);
      grad[col] = phi_over_lam * dlam + dot(g_n, dn) +
                  dPhi_dw[0] * dw[0] + dPhi_dw[1] * dw[1] + dPhi_dw[2] * dw[2] + dPhi_dw[3] * dw[3];
    }
  for (int q = 0; q < 4; ++q) {
    const NodeMap mq = vertex_nodes(S, ids[q]);
    for (int rr = 0; rr < mq.n; ++rr)
      for (int c = 0; c < 3; ++c) acc_add(gz + 3 * ((size_t)(3 * mq.node[rr] + c)), -scale * mq.w[rr] * grad[3 * q + c], S.err);
  }
}

// Friction on the lagged pairs.  Stores the 3x3 tangent Hessian Hu (scaled)
// per pair: the pair's 12x12 block is (w w^T) (x) Hu.
__global__ void k_friction(DevScene S, const double* __restrict__ xv, const double* __restrict__ xv_t, int n,
                           const int* __restrict__ f_ids, const double* __restrict__ f_w, const double* __restrict__ f_n,
                           const double* __restrict__ f_lam, double mu, double eps, double scale, int mode,
                           acc_t* __restrict__ g, double* __restrict__ f_Hu, acc_t* __restrict__ Dc,
                           const double* __restrict__ pD, acc_t* __restrict__ gdir, acc_t* __restrict__ E) {
  double e_acc = 0.0;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    int ids[4];
    double w[4];
    d3 u = mk(0, 0, 0);
    for (int q = 0; q < 4; ++q) {
      ids[q] = f_ids[4 * k + q];
      w[q] = f_w[4 * k + q];
      u = u + w[q] * (ld3(xv, ids[q]) - ld3(xv_t, ids[q]));
    }
    d3 nrm = ld3(f_n, k);
    d3 t = u - dot(nrm, u) * nrm;
    double y = sqrt(dot(t, t));
    double c = mu * f_lam[k];
    double f0 = y < eps ? -y * y * y / (3.0 * eps * eps) + y * y / eps + eps / 3.0 : y;
    e_acc = c * f0;
    if (S.E_sc) scene_energy(S, scene_of_vertex(S, ids[0]), 3, e_acc);
    if (mode >= 1) {
      double a = y < eps ? (-y / (eps * eps) + 2.0 / eps) : 1.0 / y;
      d3 gu = (c * a) * t;
      for (int q = 0; q < 4; ++q) {
        NodeMap m = vertex_nodes(S, ids[q]);
        for (int r = 0; r < m.n; ++r) {
          double ww = scale * w[q] * m.w[r];
          acc_add(g + 3 * ((size_t)(3 * m.node[r])), ww * gu.x, S.err);
          acc_add(g + 3 * ((size_t)(3 * m.node[r] + 1)), ww * gu.y, S.err);
          acc_add(g + 3 * ((size_t)(3 * m.node[r] + 2)), ww * gu.z, S.err);
        }
      }
    }
    if (mode >= 2) {
      double a = y < eps ? (-y / (eps * eps) + 2.0 / eps) : 1.0 / y;
      double bc = y < eps ? (y > 0.0 ? (-1.0 / (eps * eps)) / y : 0.0) : -1.0 / (y * y * y);
      double nv[3] = {nrm.x, nrm.y, nrm.z}, tv[3] = {t.x, t.y, t.z};
      double Hu[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          Hu[3 * i + j] = scale * c * (a * ((i == j ? 1.0 : 0.0) - nv[i] * nv[j]) + bc * tv[i] * tv[j]);
      for (int q = 0; q < 9; ++q) f_Hu[9 * k + q] = Hu[q];
      // diagonal blocks and Dirichlet term of (w w^T) (x) Hu
      NodeMap m[4];
      bool kin[4];
      d3 ud = mk(0, 0, 0);
      for (int q = 0; q < 4; ++q) {
        m[q] = vertex_nodes(S, ids[q]);
        kin[q] = S.vkind[ids[q]] == VK_KIN;
        if (kin[q]) ud = ud + w[q] * ld3(pD, ids[q] - S.nf - S.na_v);
      }
      d3 hd = mk(Hu[0] * ud.x + Hu[1] * ud.y + Hu[2] * ud.z, Hu[3] * ud.x + Hu[4] * ud.y + Hu[5] * ud.z,
                 Hu[6] * ud.x + Hu[7] * ud.y + Hu[8] * ud.z);
      for (int a_ = 0; a_ < 4; ++a_) {
        if (kin[a_] || w[a_] == 0.0) continue;
        for (int r = 0; r < m[a_].n; ++r) {
          double ww = w[a_] * m[a_].w[r];
          if (hd.x != 0.0 || hd.y != 0.0 || hd.z != 0.0) {
            acc_add(gdir + 3 * ((size_t)(3 * m[a_].node[r])), ww * hd.x, S.err);
            acc_add(gdir + 3 * ((size_t)(3 * m[a_].node[r] + 1)), ww * hd.y, S.err);
            acc_add(gdir + 3 * ((size_t)(3 * m[a_].node[r] + 2)), ww * hd.z, S.err);
          }
        }
        for (int b_ = 0; b_ < 4; ++b_) {
          if (kin[b_] || w[b_] == 0.0) continue;
          for (int r = 0; r < m[a_].n; ++r)
            for (int q = 0; q < m[b_].n; ++q) {
              if (m[a_].node[r] != m[b_].node[q]) continue;
              double ww = w[a_] * m[a_].w[r] * w[b_] * m[b_].w[q];
              for (int i = 0; i < 9; ++i) acc_add(Dc + 3 * (9 * (size_t)m[a_].node[r] + i), ww * Hu[i], S.err);
            }
        }
      }
    }
  }
  double s = block_sum(e_acc);
  if (threadIdx.x == 0) acc_add(E, s, S.err);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
// E += the exact sum of the barrier's per-pair slots (one thread; the slots are few)
__global__ void k_fold_slots(const acc_t* __restrict__ slots, acc_t* __restrict__ E) {
  if (blockIdx.x || threadIdx.x) return;
  acc_t w[3];
  acc_sum_words(slots, E_SLOTS, w);
  acc_add_words(E, w);
}

void launch_barrier(cudaStream_t st, int grid, const DevScene& S, const double* xv, const int* rec, const int* n_dev,
                    int cap, double sh, double kappa, double scale, int mode, int project, acc_t* g, double* pairH,
                    acc_t* Dc, const double* pD, acc_t* gdir, acc_t* E, unsigned long long* min_s, int hess_fp32) {
  // the energy of every pair goes into slot (pair mod E_SLOTS), folded into E afterwards: no partial sum
  // depends on the launch shape, and the slots spread the atomic traffic
  cudaMemsetAsync(S.e_slots, 0, sizeof(acc_t) * 3 * E_SLOTS, st);
  if (mode >= 2) {
    // one warp per pair: as many warps as the thread-per-pair launch had threads / 32, at least one block
    int wgrid = stride_grid(cap, BWARPS, 16);
    k_barrier_warp<<<wgrid, 32 * BWARPS, 0, st>>>(S, xv, rec, n_dev, cap, sh, kappa, scale, project, g, pairH, Dc, pD,
                                                   gdir, E, min_s, hess_fp32);
  } else {
    k_barrier<<<grid, 128, 0, st>>>(S, xv, rec, n_dev, cap, sh, kappa, scale, mode, project, g, pairH, Dc, pD, gdir,
                                    E, min_s);
  }
  k_fold_slots<<<1, 32, 0, st>>>(S.e_slots, E);
  count_launch(2);
}
void launch_friction_lag(cudaStream_t st, int grid, const DevScene& S, const double* xv, const int* rec, const int* n_dev,
                         int cap, double sh, double kappa, int* f_ids, double* f_w, double* f_n, double* f_lam,
                         int* f_rec) {
  k_friction_lag<<<grid, 128, 0, st>>>(S, xv, rec, n_dev, cap, sh, kappa, f_ids, f_w, f_n, f_lam, f_rec);
  count_launch();
}
void launch_friction_lag_adjoint(cudaStream_t st, const DevScene& S, const double* xv, const double* xv_t, int n,
                                 const int* f_ids, const int* f_rec, double sh, double mu, double eps, double scale,
                                 const double* lam_dof, acc_t* gz) {
  if (n <= 0) return;
  k_friction_lag_adjoint<<<(n + 63) / 64, 64, 0, st>>>(S, xv, xv_t, n, f_ids, f_rec, sh, mu, eps, scale, lam_dof, gz);
  count_launch();
}
void launch_friction(cudaStream_t st, const DevScene& S, const double* xv, const double* xv_t, int n, const int* f_ids,
                     const double* f_w, const double* f_n, const double* f_lam, double mu, double eps, double scale,
                     int mode, acc_t* g, double* f_Hu, acc_t* Dc, const double* pD, acc_t* gdir, acc_t* E) {
  if (n <= 0) return;
  k_friction<<<(n + 127) / 128, 128, 0, st>>>(S, xv, xv_t, n, f_ids, f_w, f_n, f_lam, mu, eps, scale, mode, g, f_Hu, Dc,
                                              pD, gdir, E);
  count_launch();
}

}  // namespace ipc
