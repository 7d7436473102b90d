// Block-Jacobi preconditioned conjugate gradients for H_FF p = rhs.
//
// H_FF is the sum of (1) the fixed-pattern BSR 3x3 matrix (inertia, elastic,
// stitch, ABD blocks), (2) the dense 12x12 vertex-space block of every active
// barrier pair and (3) the rank-structured block (w w^T) (x) Hu of every
// lagged friction pair, mapped to nodes by x = J z.  The whole solve is one
// cooperative kernel: three grid-wide barriers per iteration, dot products
// reduced per block and summed in block order by every block, so all blocks
// take identical control decisions.
#include <cooperative_groups.h>
#include <algorithm>
#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace ipc {

// Dinv_i = (BSR diagonal block + contact diagonal block)^-1
__global__ void k_dinv(int n_nodes, const int* __restrict__ diag, const double* __restrict__ val,
                       const double* __restrict__ Dc, double* __restrict__ Dinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const double* A = val + 9 * (size_t)diag[i];
  double m[9];
  for (int q = 0; q < 9; ++q) m[q] = A[q] + Dc[9 * i + q];
  double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
  double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
  double* o = Dinv + 9 * i;
  if (!(fabs(det) > 0.0)) {
    for (int q = 0; q < 9; ++q) o[q] = (q % 4 == 0 && m[q] != 0.0) ? 1.0 / m[q] : 0.0;
    return;
  }
  double id = 1.0 / det;
  o[0] = c00 * id; o[1] = (m[2] * m[7] - m[1] * m[8]) * id; o[2] = (m[1] * m[5] - m[2] * m[4]) * id;
  o[3] = c01 * id; o[4] = (m[0] * m[8] - m[2] * m[6]) * id; o[5] = (m[2] * m[3] - m[0] * m[5]) * id;
  o[6] = c02 * id; o[7] = (m[1] * m[6] - m[0] * m[7]) * id; o[8] = (m[0] * m[4] - m[1] * m[3]) * id;
}

// rhs = -(g + gdir)
__global__ void k_rhs(int n, const double* __restrict__ g, const double* __restrict__ gdir, double* __restrict__ rhs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rhs[i] = -(g[i] + gdir[i]);
}

__device__ inline double grid_total(const double* part, int nblk) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += part[b];
  __shared__ double tot;
  v = block_sum(v);
  if (threadIdx.x == 0) tot = v;
  __syncthreads();
  double r = tot;
  __syncthreads();
  return r;
}

__device__ inline d3 node_gather(const DevScene& S, const double* p, int v) {
  NodeMap m = vertex_nodes(S, v);
  d3 u = mk(0, 0, 0);
  for (int r = 0; r < m.n; ++r) u = u + m.w[r] * ld3(p, m.node[r]);
  return u;
}
__device__ inline void node_scatter(const DevScene& S, double* y, int v, d3 w) {
  NodeMap m = vertex_nodes(S, v);
  for (int r = 0; r < m.n; ++r) {
    atomicAdd(y + 3 * m.node[r], m.w[r] * w.x);
    atomicAdd(y + 3 * m.node[r] + 1, m.w[r] * w.y);
    atomicAdd(y + 3 * m.node[r] + 2, m.w[r] * w.z);
  }
}

// y += A p for the whole operator (matrix values of type M, vector p of type V,
// products and row sums in M); returns this thread's share of p^T A p in FP64.
template <typename M, typename V>
__device__ inline double apply_A(const PcgArgs& a, const M* val, const M* pairH, const M* fHu, const V* p, double* y,
                                 int tid, int nthr) {
  const DevScene& S = a.S;
  double acc = 0.0;
  for (int i = tid; i < a.n_nodes; i += nthr) {
    M s0 = M(0), s1 = M(0), s2 = M(0);
    for (int k = a.row[i]; k < a.row[i + 1]; ++k) {
      const M* A = val + 9 * (size_t)k;
      int j = a.col[k];
      M p0 = (M)p[3 * j], p1 = (M)p[3 * j + 1], p2 = (M)p[3 * j + 2];
      s0 += A[0] * p0 + A[1] * p1 + A[2] * p2;
      s1 += A[3] * p0 + A[4] * p1 + A[5] * p2;
      s2 += A[6] * p0 + A[7] * p1 + A[8] * p2;
    }
    atomicAdd(y + 3 * i, (double)s0);
    atomicAdd(y + 3 * i + 1, (double)s1);
    atomicAdd(y + 3 * i + 2, (double)s2);
    acc += (double)p[3 * i] * (double)s0 + (double)p[3 * i + 1] * (double)s1 + (double)p[3 * i + 2] * (double)s2;
  }
  int np = min(*a.n_pairs, a.cap);
  for (int k = tid; k < np; k += nthr) {
    const int* r = a.rec + 8 * k;
    const M* H = pairH + 144 * (size_t)k;
    M u[12];
    bool kin[4];
    for (int q = 0; q < 4; ++q) {
      int v = r[4 + q];
      kin[q] = S.vkind[v] == VK_KIN;
      NodeMap m = vertex_nodes(S, v);
      M ux = M(0), uy = M(0), uz = M(0);
      if (!kin[q])
        for (int t = 0; t < m.n; ++t) {
          M w = (M)m.w[t];
          ux += w * (M)p[3 * m.node[t]];
          uy += w * (M)p[3 * m.node[t] + 1];
          uz += w * (M)p[3 * m.node[t] + 2];
        }
      u[3 * q] = ux; u[3 * q + 1] = uy; u[3 * q + 2] = uz;
    }
    for (int q = 0; q < 4; ++q) {
      if (kin[q]) continue;
      M w0 = M(0), w1 = M(0), w2 = M(0);
      const M* H0 = H + 12 * (3 * q);
      for (int j = 0; j < 12; ++j) {
        w0 += H0[j] * u[j];
        w1 += H0[12 + j] * u[j];
        w2 += H0[24 + j] * u[j];
      }
      node_scatter(S, y, r[4 + q], mk((double)w0, (double)w1, (double)w2));
      acc += (double)u[3 * q] * (double)w0 + (double)u[3 * q + 1] * (double)w1 + (double)u[3 * q + 2] * (double)w2;
    }
  }
  for (int k = tid; k < a.n_fric; k += nthr) {
    const int* ids = a.f_ids + 4 * k;
    const double* w = a.f_w + 4 * k;
    const M* Hu = fHu + 9 * k;
    M U0 = M(0), U1 = M(0), U2 = M(0);
    bool kin[4];
    for (int q = 0; q < 4; ++q) {
      kin[q] = S.vkind[ids[q]] == VK_KIN;
      if (kin[q] || w[q] == 0.0) continue;
      NodeMap m = vertex_nodes(S, ids[q]);
      for (int t = 0; t < m.n; ++t) {
        M ww = (M)(w[q] * m.w[t]);
        U0 += ww * (M)p[3 * m.node[t]];
        U1 += ww * (M)p[3 * m.node[t] + 1];
        U2 += ww * (M)p[3 * m.node[t] + 2];
      }
    }
    M t0 = Hu[0] * U0 + Hu[1] * U1 + Hu[2] * U2, t1 = Hu[3] * U0 + Hu[4] * U1 + Hu[5] * U2,
      t2 = Hu[6] * U0 + Hu[7] * U1 + Hu[8] * U2;
    d3 t = mk((double)t0, (double)t1, (double)t2);
    for (int q = 0; q < 4; ++q)
      if (!kin[q] && w[q] != 0.0) node_scatter(S, y, ids[q], w[q] * t);
    acc += (double)U0 * t.x + (double)U1 * t.y + (double)U2 * t.z;
  }
  return acc;
}

// z = Dinv r for node i (Dinv of type M, z stored as V); returns r.z and r.r shares
template <typename M, typename V>
__device__ inline void precond_node(const M* Dinv, const double* r, V* z, int i, double& rz, double& rr) {
  const M* D = Dinv + 9 * i;
  M r0 = (M)r[3 * i], r1 = (M)r[3 * i + 1], r2 = (M)r[3 * i + 2];
  M z0 = D[0] * r0 + D[1] * r1 + D[2] * r2, z1 = D[3] * r0 + D[4] * r1 + D[5] * r2, z2 = D[6] * r0 + D[7] * r1 + D[8] * r2;
  z[3 * i] = (V)z0; z[3 * i + 1] = (V)z1; z[3 * i + 2] = (V)z2;
  rz += r[3 * i] * (double)z[3 * i] + r[3 * i + 1] * (double)z[3 * i + 1] + r[3 * i + 2] * (double)z[3 * i + 2];
  rr += r[3 * i] * r[3 * i] + r[3 * i + 1] * r[3 * i + 1] + r[3 * i + 2] * r[3 * i + 2];
}

// w += A u over the BSR rows, ROWG threads per row (row blocks strided among
// them, partial sums combined by shuffles); returns this thread's share of
// u^T (A_bsr u).  Every thread of the grid must call it (whole warps shuffle).
template <typename M, typename V, int ROWG>
__device__ inline double spmv_bsr(const PcgArgs& a, const M* val, const V* u, double* w, int tid, int nthr) {
  double acc = 0.0;
  int gl = threadIdx.x & (ROWG - 1);
  int group = tid / ROWG, ngroups = nthr / ROWG;
  int n_pad = ((a.n_nodes + ngroups - 1) / ngroups) * ngroups;
  for (int i = group; i < n_pad; i += ngroups) {
    M s0 = M(0), s1 = M(0), s2 = M(0);
    if (i < a.n_nodes) {
      int k1 = a.row[i + 1];
      for (int k = a.row[i] + gl; k < k1; k += ROWG) {
        const M* A = val + 9 * (size_t)k;
        int j = a.col[k];
        M p0 = (M)u[3 * j], p1 = (M)u[3 * j + 1], p2 = (M)u[3 * j + 2];
        s0 += A[0] * p0 + A[1] * p1 + A[2] * p2;
        s1 += A[3] * p0 + A[4] * p1 + A[5] * p2;
        s2 += A[6] * p0 + A[7] * p1 + A[8] * p2;
      }
    }
    for (int o = ROWG / 2; o > 0; o >>= 1) {
      s0 += __shfl_down_sync(0xffffffffu, s0, o, ROWG);
      s1 += __shfl_down_sync(0xffffffffu, s1, o, ROWG);
      s2 += __shfl_down_sync(0xffffffffu, s2, o, ROWG);
    }
    if (gl == 0 && i < a.n_nodes) {
      atomicAdd(w + 3 * i, (double)s0);
      atomicAdd(w + 3 * i + 1, (double)s1);
      atomicAdd(w + 3 * i + 2, (double)s2);
      acc += (double)u[3 * i] * (double)s0 + (double)u[3 * i + 1] * (double)s1 + (double)u[3 * i + 2] * (double)s2;
    }
  }
  return acc;
}

// Contact terms of w += A u, one warp per barrier pair and per friction pair:
// lane j < 12 gathers u for DOF j of the stencil (slot j / 3, component j % 3),
// lane r < 12 forms row r of the 12x12 block product and scatters it.
// Returns this lane's share of u^T (A_contact u).  Whole warps must call it.
template <typename M, typename V>
__device__ inline double apply_contact_warp(const PcgArgs& a, const M* pairH, const M* fHu, const V* u, double* w,
                                            int tid, int nthr) {
  const DevScene& S = a.S;
  int lane = threadIdx.x & 31;
  int warp = tid >> 5, nwarps = nthr >> 5;
  double acc = 0.0;
  int np = min(*a.n_pairs, a.cap);
  int slot = lane / 3, comp = lane % 3;
  for (int k = warp; k < np; k += nwarps) {
    const int* r = a.rec + 8 * k;
    int v = lane < 12 ? r[4 + slot] : 0;
    bool active = lane < 12 && S.vkind[v] != VK_KIN;
    M uj = M(0);
    if (active) {
      NodeMap m = vertex_nodes(S, v);
      for (int t = 0; t < m.n; ++t) uj += (M)m.w[t] * (M)u[3 * m.node[t] + comp];
    }
    const M* H = pairH + 144 * (size_t)k + 12 * (lane < 12 ? lane : 0);
    M wr = M(0);
    for (int j = 0; j < 12; ++j) {
      M uv = __shfl_sync(0xffffffffu, uj, j);
      if (lane < 12) wr += H[j] * uv;
    }
    if (active) {
      NodeMap m = vertex_nodes(S, v);
      for (int t = 0; t < m.n; ++t) atomicAdd(w + 3 * m.node[t] + comp, m.w[t] * (double)wr);
      acc += (double)uj * (double)wr;
    }
  }
  for (int k = warp; k < a.n_fric; k += nwarps) {
    const int* ids = a.f_ids + 4 * k;
    const double* wk = a.f_w + 4 * k;
    const M* Hu = fHu + 9 * k;
    int v = lane < 12 ? ids[slot] : 0;
    double wgt = lane < 12 ? wk[slot] : 0.0;
    bool active = lane < 12 && wgt != 0.0 && S.vkind[v] != VK_KIN;
    M uj = M(0);
    if (active) {
      NodeMap m = vertex_nodes(S, v);
      for (int t = 0; t < m.n; ++t) uj += (M)m.w[t] * (M)u[3 * m.node[t] + comp];
    }
    // U_c = sum over slots of w_k u_{k,c}: lanes c, c+3, c+6, c+9
    M contrib = (M)wgt * uj;
    M U0 = M(0), U1 = M(0), U2 = M(0);
    for (int q = 0; q < 4; ++q) {
      U0 += __shfl_sync(0xffffffffu, contrib, 3 * q);
      U1 += __shfl_sync(0xffffffffu, contrib, 3 * q + 1);
      U2 += __shfl_sync(0xffffffffu, contrib, 3 * q + 2);
    }
    M tc = M(0);
    if (lane < 12) tc = Hu[3 * comp] * U0 + Hu[3 * comp + 1] * U1 + Hu[3 * comp + 2] * U2;
    if (active) {
      NodeMap m = vertex_nodes(S, v);
      double y = wgt * (double)tc;
      for (int t = 0; t < m.n; ++t) atomicAdd(w + 3 * m.node[t] + comp, m.w[t] * y);
      acc += (double)uj * y;
    }
  }
  return acc;
}

// w += A u for the whole operator (BSR + barrier pairs + friction pairs); returns this thread's share of u^T A u.
template <typename M, typename V, int ROWG>
__device__ inline double apply_full(const PcgArgs& a, const M* val, const M* pairH, const M* fHu, const V* u, double* w,
                                    int tid, int nthr) {
  double acc = spmv_bsr<M, V, ROWG>(a, val, u, w, tid, nthr);
  acc += apply_contact_warp<M, V>(a, pairH, fHu, u, w, tid, nthr);
  return acc;
}

// Sums of up to three per-thread values over the block (result in every thread).
__device__ inline void block_sum3(double& a0, double& a1, double& a2) {
  __shared__ double sh3[3][32];
  __shared__ double tot3[3];
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_down_sync(0xffffffffu, a0, o);
    a1 += __shfl_down_sync(0xffffffffu, a1, o);
    a2 += __shfl_down_sync(0xffffffffu, a2, o);
  }
  int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) { sh3[0][wi] = a0; sh3[1][wi] = a1; sh3[2][wi] = a2; }
  __syncthreads();
  if (wi == 0) {
    double b0 = lane < nw ? sh3[0][lane] : 0.0, b1 = lane < nw ? sh3[1][lane] : 0.0, b2 = lane < nw ? sh3[2][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      b0 += __shfl_down_sync(0xffffffffu, b0, o);
      b1 += __shfl_down_sync(0xffffffffu, b1, o);
      b2 += __shfl_down_sync(0xffffffffu, b2, o);
    }
    if (lane == 0) { tot3[0] = b0; tot3[1] = b1; tot3[2] = b2; }
  }
  __syncthreads();
  a0 = tot3[0]; a1 = tot3[1]; a2 = tot3[2];
  __syncthreads();
}

// Totals of three partial arrays (one entry per block), identical in every block.
__device__ inline void grid_total3(const double* p0, const double* p1, const double* p2, int nblk, double& t0,
                                   double& t1, double& t2) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    a0 += p0[b];
    a1 += p1[b];
    a2 += p2[b];
  }
  block_sum3(a0, a1, a2);
  t0 = a0; t1 = a1; t2 = a2;
}

// One PCG solve in the Chronopoulos-Gear form: both dot products of an
// iteration come from one reduction point, so an iteration costs two grid
// barriers (vector update | operator application).
//   p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,  u = M^-1 r,
//   w = A u,  gamma = r.u,  delta = u.w,
//   beta = gamma / gamma_old,  alpha = gamma / (delta - beta gamma / alpha_old).
// T = double: all FP64.  T = float: FP32 operator, preconditioner, u and p;
// x, r, w, s and every dot product FP64; at FP32 convergence up to 3
// replacements r <- b - A x with the FP64 operator.
template <typename T, int ROWG>
__global__ void __launch_bounds__(256, 2) k_pcg(PcgArgs a) {
  cg::grid_group grid = cg::this_grid();
  int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  int nblk = gridDim.x;
  int n3 = 3 * a.n_nodes;
  constexpr bool F32 = sizeof(T) == 4;
  const T* val = F32 ? (const T*)a.val32 : (const T*)a.val;
  const T* pairH = F32 ? (const T*)a.pairH32 : (const T*)a.pairH;
  const T* fHu = F32 ? (const T*)a.f_Hu32 : (const T*)a.f_Hu;
  const T* Dinv = F32 ? (const T*)a.Dinv32 : (const T*)a.Dinv;
  T* pv = F32 ? (T*)a.p32 : (T*)a.p;
  T* uv = F32 ? (T*)a.z32 : (T*)a.z;
  double* w = a.y;
  double* sv = a.s;
  // partial sums: A (u.Au) is rewritten one barrier after its last read; B (r.u) and C (r.r)
  // are written in the vector phase right after the reads, so they alternate between two
  // buffers by iteration parity (a buffer is rewritten two barriers after its last read)
  double* partA = a.partial;
  auto partB = [&](int par) { return a.partial + (1 + par) * nblk; };
  auto partC = [&](int par) { return a.partial + (3 + par) * nblk; };
  // x = 0, r = b, u = M^-1 r, p = s = w = 0
  double g_l = 0.0, rr_l = 0.0;
  for (int i = tid; i < a.n_nodes; i += nthr) {
    for (int d = 0; d < 3; ++d) {
      a.x[3 * i + d] = 0.0;
      a.r[3 * i + d] = a.b[3 * i + d];
      w[3 * i + d] = 0.0;
      sv[3 * i + d] = 0.0;
      pv[3 * i + d] = T(0);
    }
    precond_node<T, T>(Dinv, a.r, uv, i, g_l, rr_l);
  }
  double zero = 0.0;
  block_sum3(g_l, rr_l, zero);
  if (threadIdx.x == 0) { partB(1)[blockIdx.x] = g_l; partC(1)[blockIdx.x] = rr_l; }
  grid.sync();
  double d_l = apply_full<T, T, ROWG>(a, val, pairH, fHu, uv, w, tid, nthr);
  double v = block_sum(d_l);
  if (threadIdx.x == 0) partA[blockIdx.x] = v;
  grid.sync();
  double gamma, rr, delta;
  grid_total3(partB(1), partC(1), partA, nblk, gamma, rr, delta);
  double bb = rr;
  double tol2 = a.rtol * a.rtol * bb;
  int it = 0, status = 0, replaced = 0;
  double alpha = 0.0, beta = 0.0;
  if (bb > 0.0) {
    if (!(delta > 0.0)) status = isfinite(delta) ? 1 : 2;
    alpha = gamma / delta;
    for (it = 0; status == 0 && it < a.max_iter; ++it) {
      // V: vector updates (node-local); w is consumed into s and cleared for the next product
      g_l = 0.0;
      rr_l = 0.0;
      for (int i = tid; i < a.n_nodes; i += nthr) {
        for (int d = 0; d < 3; ++d) {
          int q = 3 * i + d;
          double pq = (double)uv[q] + beta * (double)pv[q];
          double sq = w[q] + beta * sv[q];
          pv[q] = (T)pq;
          sv[q] = sq;
          a.x[q] += alpha * pq;
          a.r[q] -= alpha * sq;
          w[q] = 0.0;
        }
        precond_node<T, T>(Dinv, a.r, uv, i, g_l, rr_l);
      }
      const int par = it & 1;
      zero = 0.0;
      block_sum3(g_l, rr_l, zero);
      if (threadIdx.x == 0) { partB(par)[blockIdx.x] = g_l; partC(par)[blockIdx.x] = rr_l; }
      grid.sync();
      // W: w = A u and u.w
      d_l = apply_full<T, T, ROWG>(a, val, pairH, fHu, uv, w, tid, nthr);
      v = block_sum(d_l);
      if (threadIdx.x == 0) partA[blockIdx.x] = v;
      grid.sync();
      double gamma_new;
      grid_total3(partB(par), partC(par), partA, nblk, gamma_new, rr, delta);
      if (!isfinite(rr) || !isfinite(delta)) { status = 2; ++it; break; }
      if (rr <= tol2) {
        if (!F32 || replaced >= 3) { ++it; break; }
        // FP64 residual replacement and restart: r = b - A64 x
        ++replaced;
        for (int q = tid; q < n3; q += nthr) sv[q] = 0.0;
        grid.sync();
        apply_full<double, double, ROWG>(a, a.val, a.pairH, a.f_Hu, a.x, sv, tid, nthr);
        grid.sync();
        g_l = 0.0;
        rr_l = 0.0;
        for (int i = tid; i < a.n_nodes; i += nthr) {
          for (int d = 0; d < 3; ++d) {
            int q = 3 * i + d;
            a.r[q] = a.b[q] - sv[q];
            w[q] = 0.0;
            sv[q] = 0.0;
            pv[q] = T(0);
          }
          precond_node<T, T>(Dinv, a.r, uv, i, g_l, rr_l);
        }
        // this iteration's buffer: read before the two barriers above, rewritten next at it + 2
        zero = 0.0;
        block_sum3(g_l, rr_l, zero);
        if (threadIdx.x == 0) { partB(par)[blockIdx.x] = g_l; partC(par)[blockIdx.x] = rr_l; }
        grid.sync();
        d_l = apply_full<T, T, ROWG>(a, val, pairH, fHu, uv, w, tid, nthr);
        v = block_sum(d_l);
        if (threadIdx.x == 0) partA[blockIdx.x] = v;
        grid.sync();
        grid_total3(partB(par), partC(par), partA, nblk, gamma, rr, delta);
        if (rr <= tol2) { ++it; break; }
        if (!(delta > 0.0)) { status = isfinite(delta) ? 1 : 2; ++it; break; }
        beta = 0.0;
        alpha = gamma / delta;
        continue;
      }
      beta = gamma_new / gamma;
      double den = delta - beta * gamma_new / alpha;
      if (!(den > 0.0)) { status = isfinite(den) ? 1 : 2; ++it; break; }
      alpha = gamma_new / den;
      gamma = gamma_new;
    }
  } else {
    for (int i = tid; i < n3; i += nthr) a.x[i] = 0.0;
  }
  if (tid == 0) {
    a.out[0] = it;
    a.out[1] = status;
    a.out[2] = replaced;
    a.res[0] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

__global__ void k_to_float(size_t n, const double* __restrict__ src, float* __restrict__ dst, const int* n_dev,
                           int stride) {
  size_t lim = n;
  if (n_dev) lim = min(n, (size_t)(*n_dev) * (size_t)stride);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < lim; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

void launch_dinv(cudaStream_t st, int n_nodes, const int* diag, const double* val, const double* Dc, double* Dinv) {
  if (n_nodes) { k_dinv<<<(n_nodes + 255) / 256, 256, 0, st>>>(n_nodes, diag, val, Dc, Dinv); count_launch(); }
}
void launch_rhs(cudaStream_t st, int n, const double* g, const double* gdir, double* rhs) {
  if (n) { k_rhs<<<(n + 255) / 256, 256, 0, st>>>(n, g, gdir, rhs); count_launch(); }
}

int pcg_max_blocks(int threads) {
  int dev, sms, per_sm;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<double, 4>, threads, 0);
  return sms * (per_sm > 0 ? per_sm : 1);
}

int pcg_max_blocks_fp32(int threads) {
  int dev, sms, per_sm;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<float, 4>, threads, 0);
  return sms * (per_sm > 0 ? per_sm : 1);
}

template <typename T>
static void* pcg_kernel(int rowg) {
  switch (rowg) {
    case 2: return (void*)k_pcg<T, 2>;
    case 8: return (void*)k_pcg<T, 8>;
    case 16: return (void*)k_pcg<T, 16>;
    default: return (void*)k_pcg<T, 4>;
  }
}

cudaError_t launch_pcg(cudaStream_t st, int grid, int threads, const PcgArgs& a, int rowg) {
  void* args[] = {(void*)&a};
  count_launch();
  void* f = a.fp32 ? pcg_kernel<float>(rowg) : pcg_kernel<double>(rowg);
  return cudaLaunchCooperativeKernel(f, dim3(grid), dim3(threads), args, 0, st);
}

void launch_to_float(cudaStream_t st, size_t n, const double* src, float* dst, const int* n_dev, int stride) {
  if (!n) return;
  int grid = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
  k_to_float<<<grid, 256, 0, st>>>(n, src, dst, n_dev, stride);
  count_launch();
}

}  // namespace ipc
