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

// y += A p for the whole operator; returns this thread's share of p^T A p.
__device__ inline double apply_A(const PcgArgs& a, const double* p, double* y, int tid, int nthr) {
  const DevScene& S = a.S;
  double acc = 0.0;
  for (int i = tid; i < a.n_nodes; i += nthr) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = a.row[i]; k < a.row[i + 1]; ++k) {
      const double* A = a.val + 9 * (size_t)k;
      int j = a.col[k];
      double p0 = p[3 * j], p1 = p[3 * j + 1], p2 = p[3 * j + 2];
      s0 += A[0] * p0 + A[1] * p1 + A[2] * p2;
      s1 += A[3] * p0 + A[4] * p1 + A[5] * p2;
      s2 += A[6] * p0 + A[7] * p1 + A[8] * p2;
    }
    atomicAdd(y + 3 * i, s0);
    atomicAdd(y + 3 * i + 1, s1);
    atomicAdd(y + 3 * i + 2, s2);
    acc += p[3 * i] * s0 + p[3 * i + 1] * s1 + p[3 * i + 2] * s2;
  }
  int np = min(*a.n_pairs, a.cap);
  for (int k = tid; k < np; k += nthr) {
    const int* r = a.rec + 8 * k;
    const double* H = a.pairH + 144 * (size_t)k;
    double u[12];
    bool kin[4];
    for (int q = 0; q < 4; ++q) {
      int v = r[4 + q];
      kin[q] = S.vkind[v] == VK_KIN;
      d3 uq = kin[q] ? mk(0, 0, 0) : node_gather(S, p, v);
      u[3 * q] = uq.x; u[3 * q + 1] = uq.y; u[3 * q + 2] = uq.z;
    }
    for (int q = 0; q < 4; ++q) {
      if (kin[q]) continue;
      double w0 = 0.0, w1 = 0.0, w2 = 0.0;
      const double* H0 = H + 12 * (3 * q);
      for (int j = 0; j < 12; ++j) {
        w0 += H0[j] * u[j];
        w1 += H0[12 + j] * u[j];
        w2 += H0[24 + j] * u[j];
      }
      node_scatter(S, y, r[4 + q], mk(w0, w1, w2));
      acc += u[3 * q] * w0 + u[3 * q + 1] * w1 + u[3 * q + 2] * w2;
    }
  }
  for (int k = tid; k < a.n_fric; k += nthr) {
    const int* ids = a.f_ids + 4 * k;
    const double* w = a.f_w + 4 * k;
    const double* Hu = a.f_Hu + 9 * k;
    d3 U = mk(0, 0, 0);
    bool kin[4];
    for (int q = 0; q < 4; ++q) {
      kin[q] = S.vkind[ids[q]] == VK_KIN;
      if (!kin[q] && w[q] != 0.0) U = U + w[q] * node_gather(S, p, ids[q]);
    }
    d3 t = mk(Hu[0] * U.x + Hu[1] * U.y + Hu[2] * U.z, Hu[3] * U.x + Hu[4] * U.y + Hu[5] * U.z,
              Hu[6] * U.x + Hu[7] * U.y + Hu[8] * U.z);
    for (int q = 0; q < 4; ++q)
      if (!kin[q] && w[q] != 0.0) node_scatter(S, y, ids[q], w[q] * t);
    acc += dot(U, t);
  }
  return acc;
}

__global__ void k_pcg(PcgArgs a) {
  cg::grid_group grid = cg::this_grid();
  int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  int nblk = gridDim.x;
  int n3 = 3 * a.n_nodes;
  double* partA = a.partial;
  double* partB = a.partial + nblk;
  double* partC = a.partial + 2 * nblk;
  // x = 0, r = b, z = Dinv r, p = z, y = 0
  double rz_l = 0.0, bb_l = 0.0;
  for (int i = tid; i < a.n_nodes; i += nthr) {
    const double* D = a.Dinv + 9 * i;
    double r0 = a.b[3 * i], r1 = a.b[3 * i + 1], r2 = a.b[3 * i + 2];
    double z0 = D[0] * r0 + D[1] * r1 + D[2] * r2, z1 = D[3] * r0 + D[4] * r1 + D[5] * r2,
           z2 = D[6] * r0 + D[7] * r1 + D[8] * r2;
    a.x[3 * i] = 0.0; a.x[3 * i + 1] = 0.0; a.x[3 * i + 2] = 0.0;
    a.r[3 * i] = r0; a.r[3 * i + 1] = r1; a.r[3 * i + 2] = r2;
    a.z[3 * i] = z0; a.z[3 * i + 1] = z1; a.z[3 * i + 2] = z2;
    a.p[3 * i] = z0; a.p[3 * i + 1] = z1; a.p[3 * i + 2] = z2;
    a.y[3 * i] = 0.0; a.y[3 * i + 1] = 0.0; a.y[3 * i + 2] = 0.0;
    rz_l += r0 * z0 + r1 * z1 + r2 * z2;
    bb_l += r0 * r0 + r1 * r1 + r2 * r2;
  }
  double v = block_sum(rz_l);
  if (threadIdx.x == 0) partB[blockIdx.x] = v;
  v = block_sum(bb_l);
  if (threadIdx.x == 0) partC[blockIdx.x] = v;
  grid.sync();
  double rz = grid_total(partB, nblk);
  double bb = grid_total(partC, nblk);
  double tol2 = a.rtol * a.rtol * bb;
  int it = 0, status = 0;
  double rr = bb;
  if (bb > 0.0) {
    for (it = 0; it < a.max_iter; ++it) {
      // A: y = A p, partial p^T A p
      double pap_l = apply_A(a, a.p, a.y, tid, nthr);
      v = block_sum(pap_l);
      if (threadIdx.x == 0) partA[blockIdx.x] = v;
      grid.sync();
      double pap = grid_total(partA, nblk);
      if (!(pap > 0.0)) { status = isfinite(pap) ? 1 : 2; break; }
      double alpha = rz / pap;
      // B: x += alpha p, r -= alpha y, z = Dinv r, y = 0
      double rz_n = 0.0, rr_n = 0.0;
      for (int i = tid; i < a.n_nodes; i += nthr) {
        const double* D = a.Dinv + 9 * i;
        double r0 = a.r[3 * i] - alpha * a.y[3 * i];
        double r1 = a.r[3 * i + 1] - alpha * a.y[3 * i + 1];
        double r2 = a.r[3 * i + 2] - alpha * a.y[3 * i + 2];
        a.x[3 * i] += alpha * a.p[3 * i];
        a.x[3 * i + 1] += alpha * a.p[3 * i + 1];
        a.x[3 * i + 2] += alpha * a.p[3 * i + 2];
        a.r[3 * i] = r0; a.r[3 * i + 1] = r1; a.r[3 * i + 2] = r2;
        double z0 = D[0] * r0 + D[1] * r1 + D[2] * r2, z1 = D[3] * r0 + D[4] * r1 + D[5] * r2,
               z2 = D[6] * r0 + D[7] * r1 + D[8] * r2;
        a.z[3 * i] = z0; a.z[3 * i + 1] = z1; a.z[3 * i + 2] = z2;
        a.y[3 * i] = 0.0; a.y[3 * i + 1] = 0.0; a.y[3 * i + 2] = 0.0;
        rz_n += r0 * z0 + r1 * z1 + r2 * z2;
        rr_n += r0 * r0 + r1 * r1 + r2 * r2;
      }
      v = block_sum(rz_n);
      if (threadIdx.x == 0) partB[blockIdx.x] = v;
      v = block_sum(rr_n);
      if (threadIdx.x == 0) partC[blockIdx.x] = v;
      grid.sync();
      double rz_new = grid_total(partB, nblk);
      rr = grid_total(partC, nblk);
      if (!isfinite(rr)) { status = 2; ++it; break; }
      if (rr <= tol2) { ++it; break; }
      double beta = rz_new / rz;
      rz = rz_new;
      // C: p = z + beta p
      for (int i = tid; i < n3; i += nthr) a.p[i] = a.z[i] + beta * a.p[i];
      grid.sync();
    }
  } else {
    for (int i = tid; i < n3; i += nthr) a.x[i] = 0.0;
  }
  if (tid == 0) {
    a.out[0] = it;
    a.out[1] = status;
    a.res[0] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
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
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg, threads, 0);
  return sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_pcg(cudaStream_t st, int grid, int threads, const PcgArgs& a) {
  void* args[] = {(void*)&a};
  count_launch();
  return cudaLaunchCooperativeKernel((void*)k_pcg, dim3(grid), dim3(threads), args, 0, st);
}

}  // namespace ipc
