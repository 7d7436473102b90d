// Coarse level of the two-level preconditioner of the Newton system's PCG.
//
// The block-Jacobi preconditioner (3x3 diagonal blocks) removes only local
// stiffness; the error modes left after it are smooth, nearly rigid motions of
// whole regions of the soft bodies, which block Jacobi needs hundreds of
// iterations to propagate.  The coarse space holds exactly those motions: for
// every FEM row segment of the PCG launch (the rows one CTA owns, a compact
// cluster of nodes when the mesh is numbered in spatial order) the three
// translations and three small rotations about the segment's centre,
//   P_i = [ I | -[(x_i - c_a) / rho_a]x ]   (node i of aggregate a, 3 x 6),
// with rho_a the aggregate's RMS radius: the scale leaves the coarse space
// (and so the preconditioner) unchanged but gives the rotation columns the
// size of the translation columns, so that A_c is not ill-conditioned by the
// length unit alone and its FP32 copy stays positive definite,
// and the preconditioner is additive:  M^-1 = D^-1 + P (P^T A P)^-1 P^T.
// Here the Galerkin matrix A_c = P^T A P (BSR operator, barrier pair blocks
// and friction blocks) is assembled densely per independent solve and
// inverted by Gauss-Jordan elimination (A_c is symmetric positive definite,
// so no pivoting is needed); the PCG kernel applies the rows of A_c^-1 that
// belong to its own aggregate.  ABD pseudo-nodes are not in the coarse space
// (their 4x4 block grid is small and already coupled by the BSR matrix).
#include <cooperative_groups.h>
#include <algorithm>
#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace ipc {

namespace {

// centre of every aggregate (the FEM rows of a run of FEM CTAs) and the scale 1 / rho of its rotations
// (0: rotations dropped)
__global__ void k_coarse_centres(const int* __restrict__ seg, const int* __restrict__ agg_cta, int n_agg,
                                 const double* __restrict__ x, double* __restrict__ centre, double* __restrict__ rot) {
  __shared__ double c_sh[3];
  const int a = blockIdx.x;
  if (a >= n_agg) return;
  const int r0 = seg[agg_cta[2 * a]], r1 = seg[agg_cta[2 * a + 1]];
  double s0 = 0, s1 = 0, s2 = 0;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    s0 += x[3 * i];
    s1 += x[3 * i + 1];
    s2 += x[3 * i + 2];
  }
  s0 = block_sum(s0);
  __syncthreads();
  s1 = block_sum(s1);
  __syncthreads();
  s2 = block_sum(s2);
  const int n = r1 - r0;
  const double inv = n > 0 ? 1.0 / n : 0.0;
  if (threadIdx.x == 0) {
    c_sh[0] = s0 * inv;
    c_sh[1] = s1 * inv;
    c_sh[2] = s2 * inv;
  }
  __syncthreads();
  const d3 c = mk(c_sh[0], c_sh[1], c_sh[2]);
  double q = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const d3 r = ld3(x, i) - c;
    q += dot(r, r);
  }
  q = block_sum(q);
  if (threadIdx.x == 0) {
    centre[3 * a] = c.x;
    centre[3 * a + 1] = c.y;
    centre[3 * a + 2] = c.z;
    // fewer than four nodes cannot carry three independent rotations: translations only
    rot[a] = (n >= 4 && q > 0.0) ? 1.0 / sqrt(q * inv) : 0.0;
  }
}

// C = P_i^T M P_j for P = [I | -[r]x]:  [[M, -M[rj]x], [[ri]x M, -[ri]x M [rj]x]]
__device__ inline void galerkin_block(const double* M, d3 ri, d3 rj, int rot_i, int rot_j, double C[36]) {
  double Sj[9] = {0, -rj.z, rj.y, rj.z, 0, -rj.x, -rj.y, rj.x, 0};  // [rj]x
  double Si[9] = {0, -ri.z, ri.y, ri.z, 0, -ri.x, -ri.y, ri.x, 0};  // [ri]x
  double MS[9], SM[9], SMS[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double a = 0, b = 0;
      for (int k = 0; k < 3; ++k) {
        a += M[3 * r + k] * Sj[3 * k + c];
        b += Si[3 * r + k] * M[3 * k + c];
      }
      MS[3 * r + c] = a;
      SM[3 * r + c] = b;
    }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double a = 0;
      for (int k = 0; k < 3; ++k) a += SM[3 * r + k] * Sj[3 * k + c];
      SMS[3 * r + c] = a;
    }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      C[6 * r + c] = M[3 * r + c];
      C[6 * r + 3 + c] = rot_j ? -MS[3 * r + c] : 0.0;
      C[6 * (3 + r) + c] = rot_i ? SM[3 * r + c] : 0.0;
      C[6 * (3 + r) + 3 + c] = (rot_i && rot_j) ? -SMS[3 * r + c] : 0.0;
    }
}

struct CoarseAsm {
  const int* node_agg;      // (nf) aggregate of every FEM node
  const int* agg_solve;     // (n_agg) solve of every aggregate, -1 none
  const int* solve_lo;      // (n_solves) first aggregate of every solve
  const int* solve_n;       // (n_solves) coarse unknowns of every solve
  const long long* off;     // (n_solves) offset of every solve's matrix
  const double* centre;     // (n_agg, 3)
  const double* rot;        // (n_agg) 1 / rho, 0: no rotations
  const double* x;          // (nf, 3)
  acc_t* Ac;                // accumulators of the solves' matrices
  int* err;
};

__device__ inline void add_block(const CoarseAsm& C, int i, int j, const double* M) {
  const int a = C.node_agg[i], b = C.node_agg[j];
  if (a < 0 || b < 0) return;
  const int s = C.agg_solve[a];
  if (s < 0 || C.agg_solve[b] != s) return;
  const d3 ri = C.rot[a] * (ld3(C.x, i) - ld3(C.centre, a)), rj = C.rot[b] * (ld3(C.x, j) - ld3(C.centre, b));
  double B[36];
  galerkin_block(M, ri, rj, C.rot[a] != 0.0, C.rot[b] != 0.0, B);
  const int n = C.solve_n[s], lo = C.solve_lo[s];
  acc_t* dst = C.Ac + 3 * C.off[s];
  const int ra = 6 * (a - lo), cb = 6 * (b - lo);
  for (int p = 0; p < 6; ++p)
    for (int q = 0; q < 6; ++q)
      if (B[6 * p + q] != 0.0) acc_add(dst + 3 * ((size_t)(ra + p) * n + cb + q), B[6 * p + q], C.err);
}

// BSR blocks between FEM nodes
__global__ void k_coarse_bsr(CoarseAsm C, int nf, const int* __restrict__ row, const int* __restrict__ col,
                             const double* __restrict__ val) {
  const int nblk = row[nf];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nblk; k += gridDim.x * blockDim.x) {
    const int j = col[k];
    if (j >= nf) continue;
    // row of block k: the last i with row[i] <= k
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (row[mid] <= k) lo = mid; else hi = mid - 1;
    }
    add_block(C, lo, j, val + 9 * (size_t)k);
  }
}

// barrier pair blocks (vertex space 12x12) and friction blocks (w_q w_r Hu) between FEM vertices
__global__ void k_coarse_pairs(CoarseAsm C, DevScene S, const int* __restrict__ rec, const int* __restrict__ n_pairs,
                               int cap, const double* __restrict__ pairH, int n_fric, const int* __restrict__ f_ids,
                               const double* __restrict__ f_w, const double* __restrict__ f_Hu) {
  const int np = min(*n_pairs, cap);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 16 * (np + n_fric); e += gridDim.x * blockDim.x) {
    const int k = e >> 4, q = (e >> 2) & 3, r = e & 3;
    const bool fric = k >= np;
    const int kk = fric ? k - np : k;
    const int* ids = fric ? f_ids + 4 * (size_t)kk : rec + 8 * (size_t)kk + 4;
    const int vq = ids[q], vr = ids[r];
    if (S.vkind[vq] != VK_FEM || S.vkind[vr] != VK_FEM) continue;
    double M[9];
    if (fric) {
      const double ww = f_w[4 * (size_t)kk + q] * f_w[4 * (size_t)kk + r];
      if (ww == 0.0) continue;
      for (int t = 0; t < 9; ++t) M[t] = ww * f_Hu[9 * (size_t)kk + t];
    } else {
      const double* H = pairH + 144 * (size_t)kk;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[3 * a + b] = H[(3 * q + a) * 12 + 3 * r + b];
    }
    add_block(C, vq, vr, M);
  }
}

// unknowns without a mode (empty aggregates, rotations of small ones): identity rows of the assembled Ac
__global__ void k_coarse_dead(CoarseAsm C, const int* __restrict__ seg, const int* __restrict__ agg_cta, int n_agg,
                              double* __restrict__ Ac) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_agg) return;
  const int s = C.agg_solve[a];
  if (s < 0) return;
  const bool empty = seg[agg_cta[2 * a]] == seg[agg_cta[2 * a + 1]];
  const int n = C.solve_n[s], base = 6 * (a - C.solve_lo[s]);
  double* dst = Ac + C.off[s];
  for (int p = 0; p < 6; ++p)
    if (empty || (p >= 3 && !C.rot[a])) dst[(size_t)(base + p) * n + base + p] = 1.0;
}

// In-place Gauss-Jordan inversion of every solve's symmetric positive definite
// matrix (no pivoting).  Step k uses the pivot row and column as they were
// before the step (saved in buf[k & 1]); the threads that write row and column
// k + 1 also save them for the next step, so one grid barrier per step.  Rows
// are spread over the CTAs (a CTA's threads run along the row, coalesced).
// status[s] != 0: a non-positive or non-finite pivot (the solve's coarse level
// is then unusable).
__global__ void k_coarse_gj(double* __restrict__ A, const long long* __restrict__ off, const int* __restrict__ nsz,
                            const long long* __restrict__ boff, int n_solves, int nmax, double* __restrict__ buf0,
                            double* __restrict__ buf1, int* __restrict__ status) {
  cg::grid_group grid = cg::this_grid();
  // save row and column 0 of every solve
  for (int s = 0; s < n_solves; ++s) {
    const int n = nsz[s];
    const double* M = A + off[s];
    double* b = buf0 + 2 * boff[s];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      b[i] = M[(size_t)i * n];
      b[n + i] = M[i];
    }
  }
  grid.sync();
  for (int k = 0; k < nmax; ++k) {
    const double* cur = (k & 1) ? buf1 : buf0;
    double* nxt = (k & 1) ? buf0 : buf1;
    for (int s = 0; s < n_solves; ++s) {
      const int n = nsz[s];
      if (k >= n) continue;
      double* M = A + off[s];
      const double* colk = cur + 2 * boff[s];
      const double* rowk = colk + n;
      const double p = rowk[k];
      const bool ok = p > 0.0 && isfinite(p);
      if (!ok && blockIdx.x == 0 && threadIdx.x == 0) status[s] = 1;
      const double ip = ok ? 1.0 / p : 0.0;
      double* ncol = nxt + 2 * boff[s];
      double* nrow = ncol + n;
      for (int i = blockIdx.x; i < n; i += gridDim.x) {
        double* Mi = M + (size_t)i * n;
        const double ci = colk[i] * ip;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          double v;
          if (i == k) v = (j == k) ? ip : rowk[j] * ip;
          else if (j == k) v = -ci;
          else v = fma(-ci, rowk[j], Mi[j]);
          Mi[j] = v;
          if (k + 1 < n) {
            if (j == k + 1) ncol[i] = v;
            if (i == k + 1) nrow[j] = v;
          }
        }
      }
    }
    grid.sync();
  }
}

}  // namespace

void coarse_layout(const PcgPlan& P, int nf, CoarseLayout& L) {
  const int nc = P.n_fem_ctas;
  L.n_ctas = nc;
  L.n_solves = P.n_psc;
  // FEM CTAs of every solve (consecutive by construction of the plan)
  std::vector<int> lo(L.n_solves, nc), hi(L.n_solves, -1);
  for (int c = 0; c < nc; ++c) {
    const int s = P.cta_scene[c];
    if (s < 0 || s >= L.n_solves) continue;
    lo[s] = std::min(lo[s], c);
    hi[s] = std::max(hi[s], c);
  }
  L.consecutive = true;
  int largest = 0;
  for (int s = 0; s < L.n_solves; ++s) {
    for (int c = lo[s]; c <= hi[s]; ++c)
      if (P.cta_scene[c] != s) L.consecutive = false;
    largest = std::max(largest, hi[s] - lo[s] + 1);
  }
  // runs of `group` CTAs form an aggregate, so that a solve has at most COARSE_MAX_UNKNOWNS unknowns
  L.group = std::max(1, (6 * largest + COARSE_MAX_UNKNOWNS - 1) / COARSE_MAX_UNKNOWNS);
  L.cta_agg.assign(nc, -1);
  L.agg_cta.clear();
  L.agg_solve.clear();
  L.solve_lo.assign(L.n_solves, 0);
  L.solve_n.assign(L.n_solves, 0);
  for (int s = 0; s < L.n_solves; ++s) {
    L.solve_lo[s] = (int)L.agg_solve.size();
    for (int c = lo[s]; c <= hi[s]; c += L.group) {
      const int a = (int)L.agg_solve.size();
      L.agg_cta.push_back(c);
      L.agg_solve.push_back(s);
      for (int k = c; k < std::min(c + L.group, hi[s] + 1); ++k) L.cta_agg[k] = a;
    }
    L.solve_n[s] = 6 * ((int)L.agg_solve.size() - L.solve_lo[s]);
  }
  L.n_agg = (int)L.agg_solve.size();
  // closing entries: the CTA after the last of each aggregate
  std::vector<int> ends(L.n_agg + 1, nc);
  for (int a = 0; a < L.n_agg; ++a) {
    int c = L.agg_cta[a];
    while (c < nc && L.cta_agg[c] == a) ++c;
    ends[a] = c;
  }
  // agg_cta as offsets: aggregate a owns CTAs [agg_cta[a], end_a); store the ends in a second half-array
  // by making every aggregate's run end where the next one starts (runs are consecutive within a solve;
  // between solves there may be none)
  std::vector<int> starts = L.agg_cta;
  L.agg_cta.assign(2 * L.n_agg + 1, nc);
  for (int a = 0; a < L.n_agg; ++a) { L.agg_cta[2 * a] = starts[a]; L.agg_cta[2 * a + 1] = ends[a]; }
  L.node_agg.assign(nf, -1);
  for (int c = 0; c < nc; ++c)
    if (L.cta_agg[c] >= 0)
      for (int i = P.seg[c]; i < P.seg[c + 1] && i < nf; ++i) L.node_agg[i] = L.cta_agg[c];
  L.off.assign(L.n_solves, 0);
  L.boff.assign(L.n_solves, 0);
  long long o = 0, bo = 0;
  L.n_max = 0;
  for (int s = 0; s < L.n_solves; ++s) {
    const int n = L.solve_n[s];
    L.off[s] = o;
    L.boff[s] = bo;
    o += (long long)n * n;
    bo += n;
    L.n_max = std::max(L.n_max, n);
  }
  L.total = o;
  L.total_n = bo;
}

cudaError_t launch_coarse_build(cudaStream_t st, const DevScene& S, const CoarseDevLayout& D, const int* seg,
                                const double* x, const double* val, const int* rec, const int* n_pairs, int cap,
                                const double* pairH, int n_fric, const int* f_ids, const double* f_w,
                                const double* f_Hu, double* Ac, acc_t* Ac_acc, double* centre, double* rot,
                                double* gj_buf, int* status) {
  const int na = D.n_agg;
  if (na <= 0 || D.total <= 0) return cudaSuccess;
  k_coarse_centres<<<na, 128, 0, st>>>(seg, D.agg_cta, na, x, centre, rot);
  cudaError_t e = cudaMemsetAsync(Ac_acc, 0, sizeof(acc_t) * 3 * (size_t)D.total, st);
  if (e != cudaSuccess) return e;
  CoarseAsm C{D.node_agg, D.agg_solve, D.solve_lo, D.solve_n, D.off, centre, rot, x, Ac_acc, S.err};
  k_coarse_bsr<<<stride_grid(S.nnzb, 256, 8), 256, 0, st>>>(C, S.nf, S.bsr_row, S.bsr_col, val);
  k_coarse_pairs<<<stride_grid(16LL * (cap + n_fric), 256, 8), 256, 0, st>>>(C, S, rec, n_pairs, cap, pairH, n_fric,
                                                                          f_ids, f_w, f_Hu);
  launch_acc_finalize(st, (size_t)D.total, Ac_acc, nullptr, Ac);
  k_coarse_dead<<<(na + 127) / 128, 128, 0, st>>>(C, seg, D.agg_cta, na, Ac);
  count_launch(4);
  e = cudaMemsetAsync(status, 0, sizeof(int) * D.n_solves, st);
  if (e != cudaSuccess) return e;
  // Gauss-Jordan: one cooperative launch, all CTAs co-resident
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_coarse_gj, 256, 0);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(device_sms() * std::max(per_sm, 1), std::max(D.n_max, 1)));
  double* A = Ac;
  const long long* off = D.off;
  const int* nsz = D.solve_n;
  const long long* boff = D.boff;
  int ns = D.n_solves, nmax = D.n_max;
  double* b0 = gj_buf;
  double* b1 = gj_buf + 2 * D.total_n;
  void* args[] = {&A, &off, &nsz, &boff, &ns, &nmax, &b0, &b1, &status};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)k_coarse_gj, dim3(grid), dim3(256), args, 0, st);
}

}  // namespace ipc
