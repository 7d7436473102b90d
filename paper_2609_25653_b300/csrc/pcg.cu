// Block-Jacobi preconditioned conjugate gradients for H_FF p = rhs.
//
// H_FF is the sum of (1) the fixed-pattern BSR 3x3 matrix (inertia, elastic,
// stitch, ABD blocks), (2) the 12x12 vertex-space block of every active
// barrier pair and (3) the rank-structured block (w w^T) (x) Hu of every
// lagged friction pair, mapped to nodes by x = J z.
//
// The whole solve is one cooperative kernel built around three choices:
//  * owner computes: each node row of A v is formed by one group of threads
//    (a FEM node) or one CTA (the four pseudo-nodes of an ABD body).  Contact
//    pairs reach their rows through per-owner incidence lists, so no atomics
//    are needed and a row is complete inside the phase that forms it;
//  * the pipelined recurrences of Ghysels and Vanroose (2014): the matrix
//    product of iteration i does not depend on the dot products of iteration
//    i, so an iteration costs one grid-wide barrier;
//  * when they fit, every CTA keeps its rows of the operator and of the
//    preconditioner in shared memory for the whole solve.
// Dot products are reduced per CTA; every CTA writes its partial sums to R
// replicas and sums one replica in a fixed order, so all CTAs take identical
// control decisions without contending for one cache line.
#include <cooperative_groups.h>
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>
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

// ---------------------------------------------------------------------------
// contact incidence lists: for every FEM node the (pair, slot) entries whose
// rows land on it.  code = pair << 3 | friction << 2 | slot.  The rows of ABD
// pseudo-nodes take their contact part from the block lists below instead.
// ---------------------------------------------------------------------------
__device__ inline int owner_of(const DevScene& S, int v) { return S.vkind[v] == VK_FEM ? v : -1; }

template <bool FILL>
__global__ void k_incidence(DevScene S, const int* __restrict__ rec, const int* __restrict__ n_pairs, int cap,
                            int n_fric, const int* __restrict__ f_ids, const double* __restrict__ f_w,
                            int* __restrict__ cnt_or_cursor, int2* __restrict__ inc, long long inc_cap,
                            PairDesc* __restrict__ desc, int* __restrict__ err) {
  const int np = min(*n_pairs, cap);
  const long long tot = 4LL * (np + n_fric);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int k = (int)(e >> 2), q = (int)(e & 3), v, code;
    bool zero = false;
    int di;
    if (k < np) {
      v = rec[8 * (size_t)k + 4 + q];
      code = (k << 3) | q;
      di = k;
    } else {
      k -= np;
      zero = f_w[4 * (size_t)k + q] == 0.0;
      v = f_ids[4 * (size_t)k + q];
      code = (k << 3) | 4 | q;
      di = cap + k;
    }
    if (!FILL) {
      // the slot's part of the pair's gather descriptor
      PairDesc& D = desc[di];
      const int kind = zero ? VK_KIN : S.vkind[v];
      D.node[q] = kind == VK_FEM ? v : (kind == VK_ABD ? S.nf + 4 * S.vabd[v] : -1);
      if (kind == VK_ABD) {
        D.xb[q][0] = S.xbar[3 * v];
        D.xb[q][1] = S.xbar[3 * v + 1];
        D.xb[q][2] = S.xbar[3 * v + 2];
        atomicOr(&D.abd, 1 << q);
      } else {
        atomicAnd(&D.abd, ~(1 << q));
      }
    }
    if (zero) continue;
    int o = owner_of(S, v);
    if (o < 0) continue;
    int slot = atomicAdd(cnt_or_cursor + o, 1);
    if (FILL) {
      if (slot >= 0 && slot < inc_cap) inc[slot] = make_int2(code, o);
      else atomicOr(err, ERRF_INC);
    }
  }
}

// exclusive scan in place: tiles of 4096, then the tile totals, then the carries
constexpr int SCAN_TILE = 4096;
__device__ inline int block_exclusive_scan_1024(int v, int* warp_tot, int& total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = warp_tot[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  int incl = x + (w > 0 ? warp_tot[w - 1] : 0);
  total = warp_tot[31];
  __syncthreads();
  return incl - v;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(int n, int* __restrict__ a, int* __restrict__ tiles) {
  __shared__ int warp_tot[32];
  int base = blockIdx.x * SCAN_TILE + 4 * threadIdx.x;
  int v[4], s = 0;
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < n ? a[base + j] : 0;
    s += v[j];
  }
  int total;
  int ex = block_exclusive_scan_1024(s, warp_tot, total);
  for (int j = 0; j < 4; ++j) {
    if (base + j < n) a[base + j] = ex;
    ex += v[j];
  }
  if (threadIdx.x == 0) tiles[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_totals(int m, int* __restrict__ t) {
  __shared__ int warp_tot[32];
  int carry = 0;
  for (int base = 0; base < m; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < m ? t[i] : 0, total;
    int ex = block_exclusive_scan_1024(v, warp_tot, total);
    if (i < m) t[i] = ex + carry;
    carry += total;
  }
}

__global__ void k_scan_add(int n, int* __restrict__ a, const int* __restrict__ tiles) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += tiles[i / SCAN_TILE];
}

// Every owner's incidences in increasing code (pair, then friction flag, then slot) order: the fill
// appends them in the order its threads reach the cursor.  Lists are short (the contacts of one node).
__global__ void k_sort_incidence(int n_own, const int* __restrict__ inc_ptr, long long inc_cap,
                                 int2* __restrict__ inc) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_own) return;
  const long long b = inc_ptr[o], e = min((long long)inc_ptr[o + 1], inc_cap);
  for (long long i = b + 1; i < e; ++i) {
    const int2 x = inc[i];
    long long j = i - 1;
    while (j >= b && inc[j].x > x.x) {
      inc[j + 1] = inc[j];
      --j;
    }
    inc[j + 1] = x;
  }
}

size_t scan_tile_ints(size_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

void launch_scan_exclusive(cudaStream_t st, int n, int* a, int* tiles) {
  if (n <= 0) return;
  const int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  k_scan_tiles<<<ntiles, 1024, 0, st>>>(n, a, tiles);
  k_scan_totals<<<1, 1024, 0, st>>>(ntiles, tiles);
  k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(n, a, tiles);
  count_launch(3);
}

void launch_incidence(cudaStream_t st, const DevScene& S, const int* rec, const int* n_pairs, int cap, int n_fric,
                      const int* f_ids, const double* f_w, int* inc_ptr, int* cursor, int* tiles, int2* inc,
                      long long inc_cap, PairDesc* desc, int* err) {
  const int n_own = S.nf + S.nab;
  const int n = n_own + 1;
  cudaMemsetAsync(inc_ptr, 0, sizeof(int) * n, st);
  int grid = stride_grid(4LL * (cap + n_fric), 256, 8);
  k_incidence<false><<<grid, 256, 0, st>>>(S, rec, n_pairs, cap, n_fric, f_ids, f_w, inc_ptr, nullptr, 0, desc, err);
  int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  k_scan_tiles<<<ntiles, 1024, 0, st>>>(n, inc_ptr, tiles);
  k_scan_totals<<<1, 1024, 0, st>>>(ntiles, tiles);
  k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(n, inc_ptr, tiles);
  cudaMemcpyAsync(cursor, inc_ptr, sizeof(int) * n_own, cudaMemcpyDeviceToDevice, st);
  k_incidence<true><<<grid, 256, 0, st>>>(S, rec, n_pairs, cap, n_fric, f_ids, f_w, cursor, inc, inc_cap, desc, err);
  k_sort_incidence<<<(n_own + 127) / 128, 128, 0, st>>>(n_own, inc_ptr, inc_cap, inc);
  for (int k = 0; k < 6; ++k) count_launch();
}

// ---------------------------------------------------------------------------
// ABD bodies in contact.  For each pair, the part of J^T H J that couples the
// pseudo-nodes of one body with themselves is added into that body's 4x4 BSR
// grid, and the part that couples them with any other node becomes a list of
// 3x3 blocks per body (entry code = column node << 2 | pseudo-node row t; the
// rows t = 0..3 of one column are consecutive, so t = (entry - first entry of
// the body) mod 4), so that the ABD rows of the PCG need one gather per block.  Once per Newton
// iteration, after the pair Hessians and before the preconditioner.
// ---------------------------------------------------------------------------
struct PairSlots {
  int n;          // slots (4)
  int kind[4];    // VK_FEM / VK_ABD / VK_KIN, or -1 for a zero-weight friction slot
  int node[4];    // FEM node, or first pseudo-node of the ABD body
  int body[4];    // ABD body or -1
  double w[4][4]; // pseudo-node weights (1, xbar) of ABD slots
};

__device__ inline void pair_slots(const DevScene& S, const int* ids, const double* fw, PairSlots& P) {
  P.n = 4;
  for (int q = 0; q < 4; ++q) {
    const int v = ids[q];
    P.body[q] = -1;
    P.node[q] = -1;
    if (fw && fw[q] == 0.0) { P.kind[q] = -1; continue; }
    const int k = S.vkind[v];
    P.kind[q] = k;
    if (k == VK_FEM) {
      P.node[q] = v;
    } else if (k == VK_ABD) {
      const int b = S.vabd[v];
      P.body[q] = b;
      P.node[q] = S.nf + 4 * b;
      P.w[q][0] = 1.0;
      P.w[q][1] = S.xbar[3 * v];
      P.w[q][2] = S.xbar[3 * v + 1];
      P.w[q][3] = S.xbar[3 * v + 2];
    }
  }
}

// 3x3 block (q, j) of a pair: rows 3q.., columns 3j.. of its 12x12 (barrier) or w_q w_j Hu (friction)
__device__ inline void pair_block(const double* H, const double* fw, const double* Hu, int q, int j, double B[9]) {
  if (H) {
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) B[3 * r + c] = H[(3 * q + r) * 12 + 3 * j + c];
  } else {
    const double ww = fw[q] * fw[j];
    for (int i = 0; i < 9; ++i) B[i] = ww * Hu[i];
  }
}

// The list of a body is the concatenation of its chunks (the entries one pair adds for that body) in
// (pair, first slot) order: the counting pass writes every chunk's key (body, pair, slot) and size, the
// keys are sorted, and the scan of the sizes in sorted order gives every chunk its position.
template <bool FILL>
__global__ void k_abd_contact(DevScene S, const int* __restrict__ rec, const int* __restrict__ n_pairs, int cap,
                              const double* __restrict__ pairH, int n_fric, const int* __restrict__ f_ids,
                              const double* __restrict__ f_w, const double* __restrict__ f_Hu, int* __restrict__ cnt,
                              AbdChunks C, int* __restrict__ ent, double* __restrict__ entv, long long ent_cap,
                              acc_t* __restrict__ Hval, int* __restrict__ err) {
  const int np = min(*n_pairs, cap);
  if (!FILL && blockIdx.x == 0 && threadIdx.x == 0) *C.n = 4 * (np + n_fric);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < np + n_fric; e += gridDim.x * blockDim.x) {
    const bool fric = e >= np;
    const int k = fric ? e - np : e;
    const int* ids = fric ? f_ids + 4 * (size_t)k : rec + 8 * (size_t)k + 4;
    const double* fw = fric ? f_w + 4 * (size_t)k : nullptr;
    const double* H = fric ? nullptr : pairH + 144 * (size_t)k;
    const double* Hu = fric ? f_Hu + 9 * (size_t)k : nullptr;
    PairSlots P;
    pair_slots(S, ids, fw, P);
    for (int q0 = 0; q0 < 4; ++q0) {
      const int b = P.body[q0];
      const int chunk = 4 * e + q0;
      if (!FILL) {
        C.keys[chunk] = ~0ull;  // no chunk: sorted behind every body's chunks
        C.idx[chunk] = chunk;
        C.size[chunk] = 0;
      }
      if (b < 0) continue;
      bool first = true;
      for (int q = 0; q < q0; ++q) first = first && P.body[q] != b;
      if (!first) continue;  // body b handled at its first slot
      // columns of the list: FEM slots (one node each) and other ABD bodies (four pseudo-nodes each)
      int count = 0;
      for (int j = 0; j < 4; ++j) {
        if (P.kind[j] == VK_FEM) count += 4;
        if (P.kind[j] == VK_ABD && P.body[j] != b) {
          bool fb = true;
          for (int jj = 0; jj < j; ++jj) fb = fb && P.body[jj] != P.body[j];
          if (fb) count += 16;
        }
      }
      if (!FILL) {
        if (count) {
          atomicAdd(cnt + b, count);
          C.keys[chunk] = ((unsigned long long)b << (C.pair_bits + 2)) | ((unsigned long long)e << 2) | q0;
          C.size[chunk] = count;
        }
        continue;
      }
      double B[9];
      // same-body part into the BSR grid
      for (int t = 0; t < 4; ++t)
        for (int u = 0; u < 4; ++u) {
          double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
          for (int q = 0; q < 4; ++q) {
            if (P.body[q] != b) continue;
            for (int j = 0; j < 4; ++j) {
              if (P.body[j] != b) continue;
              pair_block(H, fw, Hu, q, j, B);
              const double ww = P.w[q][t] * P.w[j][u];
              for (int i = 0; i < 9; ++i) acc[i] += ww * B[i];
            }
          }
          acc_t* dst = Hval + 27 * (size_t)S.abd_blk[16 * b + 4 * t + u];
          for (int i = 0; i < 9; ++i) acc_add(dst + 3 * i, acc[i], S.err);
        }
      if (!count) continue;
      int pos = C.pos[chunk];
      if (pos < 0 || pos + count > ent_cap) { atomicOr(err, ERRF_ABD); continue; }
      for (int j = 0; j < 4; ++j) {
        if (P.kind[j] == VK_FEM) {
          for (int t = 0; t < 4; ++t) {
            double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int q = 0; q < 4; ++q) {
              if (P.body[q] != b) continue;
              pair_block(H, fw, Hu, q, j, B);
              for (int i = 0; i < 9; ++i) acc[i] += P.w[q][t] * B[i];
            }
            ent[pos] = (P.node[j] << 2) | t;
            for (int i = 0; i < 9; ++i) entv[9 * (size_t)pos + i] = acc[i];
            ++pos;
          }
        } else if (P.kind[j] == VK_ABD && P.body[j] != b) {
          bool fb = true;
          for (int jj = 0; jj < j; ++jj) fb = fb && P.body[jj] != P.body[j];
          if (!fb) continue;
          const int b2 = P.body[j];
          for (int u = 0; u < 4; ++u)
            for (int t = 0; t < 4; ++t) {  // t innermost: entry e of body b has t = (e - ptr[b]) & 3
              double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
              for (int q = 0; q < 4; ++q) {
                if (P.body[q] != b) continue;
                for (int jj = 0; jj < 4; ++jj) {
                  if (P.body[jj] != b2) continue;
                  pair_block(H, fw, Hu, q, jj, B);
                  const double ww = P.w[q][t] * P.w[jj][u];
                  for (int i = 0; i < 9; ++i) acc[i] += ww * B[i];
                }
              }
              ent[pos] = ((S.nf + 4 * b2 + u) << 2) | t;
              for (int i = 0; i < 9; ++i) entv[9 * (size_t)pos + i] = acc[i];
              ++pos;
            }
        }
      }
    }
  }
}

// positions of the sorted chunks: scan[i] = size of sorted chunk i (0 past the count), then pos[chunk] = scan
__global__ void k_chunk_sizes(AbdChunks C, int bound) {
  const int n = *C.n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bound; i += gridDim.x * blockDim.x)
    C.scan[i] = i < n ? C.size[C.idx[i]] : 0;
}
__global__ void k_chunk_pos(AbdChunks C) {
  const int n = *C.n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) C.pos[C.idx[i]] = C.scan[i];
}

// Merge of a body's entries with equal code (column node, row): the raw list holds one entry per pair and
// slot; sorted by (body, code) (stable: chunk order within a code) and summed run by run in that order.
__global__ void k_ent_keys(int nab, const int* __restrict__ ptr, const int* __restrict__ ent, int code_bits,
                           long long ent_cap, unsigned long long* __restrict__ keys, int* __restrict__ idx) {
  const int n = (int)min((long long)ptr[nab], ent_cap);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int lo = 0, hi = nab - 1;  // body: the last b with ptr[b] <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ptr[mid] <= e) lo = mid; else hi = mid - 1;
    }
    keys[e] = ((unsigned long long)lo << code_bits) | (unsigned)ent[e];
    idx[e] = e;
  }
}
__global__ void k_ent_heads(const int* __restrict__ n_dev, long long cap, int bound,
                            const unsigned long long* __restrict__ keys, int* __restrict__ head) {
  const int n = (int)min((long long)*n_dev, cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bound; i += gridDim.x * blockDim.x)
    head[i] = (i < n && (i == 0 || keys[i] != keys[i - 1])) ? 1 : 0;
}
__global__ void k_ent_merge(const int* __restrict__ n_dev, long long cap, int code_bits,
                            const unsigned long long* __restrict__ keys, const int* __restrict__ idx,
                            const int* __restrict__ pos, const double* __restrict__ val_raw, int* __restrict__ ent,
                            double* __restrict__ val, int* __restrict__ body_cnt) {
  const int n = (int)min((long long)*n_dev, cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i > 0 && keys[i] == keys[i - 1]) continue;
    double sum[9];
    for (int q = 0; q < 9; ++q) sum[q] = 0.0;
    int j = i;
    do {
      const double* v = val_raw + 9 * (size_t)idx[j];
      for (int q = 0; q < 9; ++q) sum[q] += v[q];
      ++j;
    } while (j < n && keys[j] == keys[i]);
    const int p = pos[i];
    ent[p] = (int)(keys[i] & ((1ull << code_bits) - 1ull));
    for (int q = 0; q < 9; ++q) val[9 * (size_t)p + q] = sum[q];
    atomicAdd(body_cnt + (int)(keys[i] >> code_bits), 1);
  }
}

void launch_abd_contact(cudaStream_t st, const DevScene& S, const int* rec, const int* n_pairs, int cap,
                        const double* pairH, int n_fric, const int* f_ids, const double* f_w, const double* f_Hu,
                        int* abd_ptr, const AbdChunks& C, int* ent, double* entv, long long ent_cap, acc_t* Hval,
                        acc_t* Dc, int* err) {
  if (S.nab == 0) return;
  // the diagonal contact blocks of the pseudo-nodes go into the BSR grid with the rest of the same-body part
  cudaMemsetAsync(Dc + 27 * (size_t)S.nf, 0, sizeof(acc_t) * 108 * (size_t)S.nab, st);
  cudaMemsetAsync(abd_ptr, 0, sizeof(int) * (S.nab + 1), st);
  const int bound = 4 * (cap + n_fric);  // chunk slots of the largest list this launch can see
  const int grid = stride_grid((long long)cap + n_fric, 128, 8);
  k_abd_contact<false><<<grid, 128, 0, st>>>(S, rec, n_pairs, cap, pairH, n_fric, f_ids, f_w, f_Hu, abd_ptr, C,
                                             nullptr, nullptr, 0, nullptr, err);
  k_scan_totals<<<1, 1024, 0, st>>>(S.nab + 1, abd_ptr);
  launch_sort_u64(st, C.n, bound, C.key_bits, C.keys, C.idx, C.keys_tmp, C.idx_tmp, C.hist, C.tiles);
  k_chunk_sizes<<<stride_grid(bound, 256, 8), 256, 0, st>>>(C, bound);
  launch_scan_exclusive(st, bound, C.scan, C.tiles);
  k_chunk_pos<<<stride_grid(bound, 256, 8), 256, 0, st>>>(C);
  k_abd_contact<true><<<grid, 128, 0, st>>>(S, rec, n_pairs, cap, pairH, n_fric, f_ids, f_w, f_Hu, nullptr, C,
                                            C.ent_raw, C.val_raw, ent_cap, Hval, err);
  // merge equal codes into the lists the PCG reads
  const int eb = (int)ent_cap;
  const int egrid = stride_grid(eb, 256, 8);
  k_ent_keys<<<egrid, 256, 0, st>>>(S.nab, abd_ptr, C.ent_raw, C.code_bits, ent_cap, C.ekeys, C.eidx);
  launch_sort_u64(st, abd_ptr + S.nab, eb, C.ekey_bits, C.ekeys, C.eidx, C.ekeys_tmp, C.eidx_tmp, C.ehist, C.etiles);
  k_ent_heads<<<egrid, 256, 0, st>>>(abd_ptr + S.nab, ent_cap, eb, C.ekeys, C.ehead);
  launch_scan_exclusive(st, eb, C.ehead, C.etiles);
  cudaMemsetAsync(C.body_cnt, 0, sizeof(int) * (S.nab + 1), st);
  k_ent_merge<<<egrid, 256, 0, st>>>(abd_ptr + S.nab, ent_cap, C.code_bits, C.ekeys, C.eidx, C.ehead, C.val_raw, ent,
                                     entv, C.body_cnt);
  k_scan_totals<<<1, 1024, 0, st>>>(S.nab + 1, C.body_cnt);
  cudaMemcpyAsync(abd_ptr, C.body_cnt, sizeof(int) * (S.nab + 1), cudaMemcpyDeviceToDevice, st);
  count_launch(9);
}

// ---------------------------------------------------------------------------
// operator in the CTA-major layout: the blocks of segment s (rows seg[s] ..
// seg[s+1]) are stored from 9 k0 on as nine planes of nloc values (value q of
// block k0 + kk at 9 k0 + q nloc + kk), so that consecutive threads read
// consecutive addresses and a CTA's rows form one contiguous range.
// ---------------------------------------------------------------------------
template <typename M>
__global__ void k_layout(const int* __restrict__ seg, const int* __restrict__ row, const double* __restrict__ src,
                         M* __restrict__ dst) {
  int s = blockIdx.x;
  int k0 = row[seg[s]], k1 = row[seg[s + 1]];
  int nloc = k1 - k0;
  const double* in = src + 9 * (size_t)k0;
  M* out = dst + 9 * (size_t)k0;
  for (int idx = threadIdx.x; idx < 9 * nloc; idx += blockDim.x) {
    int q = idx / nloc, kk = idx - q * nloc;
    out[idx] = (M)in[9 * kk + q];
  }
}

void launch_layout(cudaStream_t st, int n_seg, const int* seg, const int* row, const double* src, void* dst, int fp32) {
  if (n_seg <= 0) return;
  if (fp32) k_layout<float><<<n_seg, 256, 0, st>>>(seg, row, src, (float*)dst);
  else k_layout<double><<<n_seg, 256, 0, st>>>(seg, row, src, (double*)dst);
  count_launch();
}

// ---------------------------------------------------------------------------
// the solver kernel
// ---------------------------------------------------------------------------
template <typename T>
struct Vecs {
  T *r, *u, *w, *m0, *m1, *z, *q, *s, *p;
};

// value q of local block kk: base[q * sq + kk * sk]
template <typename M>
struct OpView {
  const M* base;
  int sq, sk;
};

// Index validation (PcgArgs::check): records the first failing site and
// tells the caller to skip the access.
__device__ inline bool pcg_ok(const PcgArgs& a, bool cond, int site) {
  if (a.check == nullptr || cond) return true;
  atomicCAS(a.check, 0, site);
  return false;
}

// v at a pair slot through its gather descriptor (x = J z; zero for kinematic slots)
template <typename V, typename A>
__device__ inline void gather_slot(const PairDesc& D, int j, const V* v, A& g0, A& g1, A& g2) {
  const int n = D.node[j];
  if (n < 0) { g0 = g1 = g2 = A(0); return; }
  const V* b = v + 3 * (size_t)n;
  g0 = (A)b[0]; g1 = (A)b[1]; g2 = (A)b[2];
  if (D.abd & (1 << j)) {
    const A x0 = (A)D.xb[j][0], x1 = (A)D.xb[j][1], x2 = (A)D.xb[j][2];
    g0 = fma(x0, (A)b[3], fma(x1, (A)b[6], fma(x2, (A)b[9], g0)));
    g1 = fma(x0, (A)b[4], fma(x1, (A)b[7], fma(x2, (A)b[10], g1)));
    g2 = fma(x0, (A)b[5], fma(x1, (A)b[8], fma(x2, (A)b[11], g2)));
  }
}

// rows (3 slot .. 3 slot + 2) of one contact block applied to v (block values
// stored as M, products and sums in A)
template <typename M, typename V, typename A>
__device__ inline void contact_rows(const PcgArgs& a, const M* pairH, const M* fHu, const V* v, int code, A& y0, A& y1,
                                    A& y2) {
  const int k = code >> 3, q = code & 3;
  const bool fric = code & 4;
  if (!pcg_ok(a, fric ? (k >= 0 && k < a.n_fric) : (k >= 0 && k < a.cap), fric ? 5 : 3)) {
    y0 = y1 = y2 = A(0);
    return;
  }
  const PairDesc& D = a.desc[fric ? (size_t)a.cap + k : (size_t)k];
  A g[4][3];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (!pcg_ok(a, D.node[j] < a.n_nodes, 4)) { g[j][0] = g[j][1] = g[j][2] = A(0); continue; }
    gather_slot<V, A>(D, j, v, g[j][0], g[j][1], g[j][2]);
  }
  if (!fric) {
    const M* H = pairH + 144 * (size_t)k + 36 * q;
    A t0 = A(0), t1 = A(0), t2 = A(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      t0 = fma((A)H[3 * j], g[j][0], fma((A)H[3 * j + 1], g[j][1], fma((A)H[3 * j + 2], g[j][2], t0)));
      t1 = fma((A)H[12 + 3 * j], g[j][0], fma((A)H[12 + 3 * j + 1], g[j][1], fma((A)H[12 + 3 * j + 2], g[j][2], t1)));
      t2 = fma((A)H[24 + 3 * j], g[j][0], fma((A)H[24 + 3 * j + 1], g[j][1], fma((A)H[24 + 3 * j + 2], g[j][2], t2)));
    }
    y0 = t0; y1 = t1; y2 = t2;
    return;
  }
  const double* w = a.f_w + 4 * (size_t)k;
  const M* Hu = fHu + 9 * (size_t)k;
  A U0 = A(0), U1 = A(0), U2 = A(0);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const A wj = (A)w[j];
    U0 = fma(wj, g[j][0], U0); U1 = fma(wj, g[j][1], U1); U2 = fma(wj, g[j][2], U2);
  }
  const A wq = (A)w[q];
  y0 = wq * fma((A)Hu[0], U0, fma((A)Hu[1], U1, (A)Hu[2] * U2));
  y1 = wq * fma((A)Hu[3], U0, fma((A)Hu[4], U1, (A)Hu[5] * U2));
  y2 = wq * fma((A)Hu[6], U0, fma((A)Hu[7], U1, (A)Hu[8] * U2));
}

// ---------------------------------------------------------------------------
// Reductions.  FP64 issue slots are scarce on this part (2 FMA / clock / SM),
// so every sum over the CTA goes through shared memory and one warp: each
// thread stores its values, warp 0 adds them in a fixed order (8 per lane and
// value), then 5 shuffle levels.
// ---------------------------------------------------------------------------
constexpr int PCG_THREADS_MAX = 256;
constexpr int PCG_REPLICAS = PCG_REPLICA_COUNT;

static_assert(PCG_SCENES_MAX <= PCG_THREADS_MAX, "one decision thread per scene");
struct Shared {
  union {
    double vals[6][PCG_THREADS_MAX];  // per-thread values of a CTA sum
    double tot[3][PCG_SCENES_MAX];    // per-scene totals (several solves)
  };
  double red[8][12];                // per-warp sums of the ABD rows
  double out[12];                   // results, read by every thread
  double scal[4];                   // scalars of an iteration (the scene's decision thread -> all)
  int action;
  unsigned long long agg[4];        // end of the solve: maxima over the scenes
};

// Sum over the CTA of N <= 6 per-thread values of type T; results in
// sh.out[0..N) (as FP64) for every thread.  Only the first `active` threads
// may hold non-zero values (the others are left out, which changes no bit).
// FP64: a pairwise tree over the thread index, all N values at once: at width
// w, (value j, slot t < w) adds slot t + w, and the N w additions of a level
// are shared out over every thread.  This part issues about 2 FP64 lanes per
// clock per SM, so a warp-wide FP64 add holds its sub-partition's FP64 unit
// for dozens of cycles: left to one warp (8 adds per lane, then 5 shuffle
// levels: 13 warp-wide adds per value on one sub-partition) the sums of an
// iteration were a large part of its critical path; the tree issues about
// 255 useful lane additions per value over all four sub-partitions.
// FP32: warp 0 adds 8 values per lane, then 5 shuffle levels.
template <int N, typename T>
__device__ inline void cta_sum(const T (&v)[N], Shared& sh, int active = PCG_THREADS_MAX) {
  T (*vals)[PCG_THREADS_MAX] = reinterpret_cast<T (*)[PCG_THREADS_MAX]>(&sh.vals[0][0]);
  if constexpr (sizeof(T) == 8) {
    const int nt = blockDim.x;
    active = max(1, min(active, nt));
    int w = 1;
    while (w < active) w <<= 1;  // w <= PCG_THREADS_MAX
    for (int t = threadIdx.x; t < w; t += nt)
#pragma unroll
      for (int j = 0; j < N; ++j) vals[j][t] = (t == (int)threadIdx.x && t < active) ? v[j] : T(0);
    __syncthreads();
    for (int lw = 31 - __clz(w) - 1; lw >= 0; --lw) {
      const int h = 1 << lw;
      for (int f = threadIdx.x; f < N * h; f += nt) {
        const int j = f >> lw, t = f & (h - 1);
        vals[j][t] += vals[j][t + h];
      }
      __syncthreads();
    }
    if (threadIdx.x < N) sh.out[threadIdx.x] = (double)vals[threadIdx.x][0];
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) vals[j][threadIdx.x] = v[j];
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        T t = T(0);
        for (int k = lane; k < (int)blockDim.x; k += 32) t += vals[j][k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) sh.out[j] = (double)t;
      }
    }
  }
  __syncthreads();
}

// Sum over the CTAs of 3 partial sums of type T (one replica [3][grid]):
// every CTA adds them in the same order, so all CTAs hold bit-identical
// totals.  The loads of the first 2 x blockDim partials are issued early.
template <typename T>
struct Partials {
  T v[3][2];
};
template <typename T>
__device__ inline void load_partials(const T* rep, int nblk, Partials<T>& P) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int b = threadIdx.x + j * blockDim.x;
    const bool in = b < nblk;
    P.v[0][j] = in ? rep[b] : T(0);
    P.v[1][j] = in ? rep[nblk + b] : T(0);
    P.v[2][j] = in ? rep[2 * nblk + b] : T(0);
  }
}

// This CTA's 3 partial sums, written to every replica.
template <typename T>
__device__ inline void write_partials(T* rep0 /* replica 0 of this parity, [3][grid] */, size_t rep_stride, int nblk,
                                      Shared& sh, const T (&v)[3], int active = PCG_THREADS_MAX) {
  cta_sum<3, T>(v, sh, active);
  if (threadIdx.x < 3 * PCG_REPLICAS) {
    int rep = threadIdx.x / 3, j = threadIdx.x % 3;
    rep0[rep * rep_stride + (size_t)j * nblk + blockIdx.x] = (T)sh.out[j];
  }
  __syncthreads();
}

// Totals of N per-CTA values for every solve, in a fixed order so that every
// CTA holds bit-identical totals.  One solve: the CTA sum over all CTAs into
// sh.out (the first 2 x blockDim values may already be in P); several: one
// thread per value and scene over that scene's CTAs into sh.tot[j][s].  Every thread must
// call it; read the results with scene_total.
template <int N, typename T>
__device__ inline void scene_totals(const PcgArgs& a, const T* rep /* [N][grid] */, int nblk, Shared& sh,
                                    const Partials<T>* P) {
  if (a.n_psc == 1) {
    T v[N];
    int start = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = T(0);
    if (P) {
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = P->v[j][0] + P->v[j][1];
      start = 2 * blockDim.x;
    }
    for (int b = threadIdx.x + start; b < nblk; b += blockDim.x) {
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] += rep[(size_t)j * nblk + b];
    }
    cta_sum<N, T>(v, sh);
    return;
  }
  // one thread per (value, scene) adds the scene's few CTA values in CTA order (a warp per scene with a
  // shuffle tree per value issued far more FP64 adds than the sums need, on few sub-partitions)
  for (int idx = threadIdx.x; idx < N * a.n_psc; idx += blockDim.x) {
    const int j = idx / a.n_psc, sc = idx - j * a.n_psc;
    const int k0 = a.sc_ptr[sc], k1 = a.sc_ptr[sc + 1];
    T v = T(0);
    for (int k = k0; k < k1; ++k) v += rep[(size_t)j * nblk + a.sc_cta[k]];
    sh.tot[j][sc] = (double)v;
  }
  __syncthreads();
}
__device__ inline double scene_total(const PcgArgs& a, const Shared& sh, int j, int sc) {
  return a.n_psc == 1 ? sh.out[j] : sh.tot[j][sc];
}

// ---------------------------------------------------------------------------
// Coarse level (coarse.cu builds it): the aggregate of a FEM CTA is its row
// segment; P_i = [I | -[x_i - c]x] maps the aggregate's 6 rigid-body
// coordinates to node i.
// ---------------------------------------------------------------------------
// This CTA's part of P^T v: its rows r0..r1 (of aggregate agg), v_i from
// get(i, v0, v1, v2), into co.part[6 cta ..] (agg < 0: nothing).  Every
// thread of the CTA must call it.
template <typename G>
__device__ inline void coarse_restrict(const PcgArgs& a, int agg, int r0, int r1, Shared& sh, G&& get) {
  double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (agg >= 0) {
    const d3 c = ld3(a.co.centre, agg);
    const double rs = a.co.rot[agg];
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double v0, v1, v2;
      get(i, v0, v1, v2);
      t[0] += v0; t[1] += v1; t[2] += v2;
      if (rs != 0.0) {
        const d3 r = rs * (ld3(a.co.x, i) - c);
        t[3] = fma(r.y, v2, fma(-r.z, v1, t[3]));
        t[4] = fma(r.z, v0, fma(-r.x, v2, t[4]));
        t[5] = fma(r.x, v1, fma(-r.y, v0, t[5]));
      }
    }
  }
  cta_sum<6, double>(t, sh, agg >= 0 ? r1 - r0 : 1);
  if (threadIdx.x < 6 && agg >= 0) a.co.part[6 * (size_t)blockIdx.x + threadIdx.x] = sh.out[threadIdx.x];
  __syncthreads();
}

// The rows of the coarse inverse that belong to aggregate agg (solve s) times
// the solve's restricted vector (every aggregate's value is the sum of its
// CTAs' parts): 6 values into res (every thread).  M: the precision of the
// stored inverse and of the products.  Every thread must call it.
template <typename M>
__device__ inline void coarse_own_t(const PcgArgs& a, const M* inv, int agg, int s, Shared& sh, double res[6],
                                    const M* rows) {
  M acc[6] = {M(0), M(0), M(0), M(0), M(0), M(0)};
  if (agg >= 0 && s >= 0) {
    const int n = a.co.solve_n[s], lo = a.co.solve_lo[s];
    const M* R = rows ? rows : inv + a.co.off[s] + (size_t)6 * (agg - lo) * n;
    // the restricted values of this thread's unknowns first (independent loads), then the products
    constexpr int PER = (COARSE_MAX_UNKNOWNS + PCG_THREADS_MAX - 1) / PCG_THREADS_MAX;
    double v[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int j = threadIdx.x + q * blockDim.x;
      v[q] = 0.0;
      if (j < n) {
        const int b = lo + j / 6, k6 = j - 6 * (j / 6);
        const int c0 = a.co.agg_cta[2 * b], c1 = a.co.agg_cta[2 * b + 1];
        for (int c = c0; c < c1; ++c) v[q] += a.co.part[6 * (size_t)c + k6];
      }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int j = threadIdx.x + q * blockDim.x;
      if (j < n) {
        const M vj = (M)v[q];
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] = fma(R[(size_t)k * n + j], vj, acc[k]);
      }
    }
  }
  const double t[6] = {(double)acc[0], (double)acc[1], (double)acc[2], (double)acc[3], (double)acc[4], (double)acc[5]};
  cta_sum<6, double>(t, sh, (agg >= 0 && s >= 0) ? a.co.solve_n[s] : 1);
#pragma unroll
  for (int k = 0; k < 6; ++k) res[k] = sh.out[k];
  __syncthreads();
}
// rows: the aggregate's six rows staged in shared memory (coarse_stage), or null
__device__ inline void coarse_own(const PcgArgs& a, int agg, int s, Shared& sh, double res[6], const void* rows) {
  if (a.co.inv64) coarse_own_t<double>(a, a.co.inv64, agg, s, sh, res, (const double*)rows);
  else coarse_own_t<float>(a, a.co.inv32, agg, s, sh, res, (const float*)rows);
}

// The six rows of the coarse inverse that belong to this CTA's aggregate, copied into the dynamic shared
// memory at a.co.smem_off once per solve (they stay fixed during the solve); returns them, or null when
// they are read from global memory.  Every thread must call it.
__device__ inline const void* coarse_stage(const PcgArgs& a, int agg, int s, unsigned char* dyn) {
  if (a.co.inv32 == nullptr || a.co.smem_off < 0) return nullptr;
  const void* out = nullptr;
  if (agg >= 0 && s >= 0) {
    const int n = a.co.solve_n[s], lo = a.co.solve_lo[s];
    const size_t first = a.co.off[s] + (size_t)6 * (agg - lo) * n;
    if (a.co.inv64) {
      double* d = reinterpret_cast<double*>(dyn + a.co.smem_off);
      for (int i = threadIdx.x; i < 6 * n; i += blockDim.x) d[i] = a.co.inv64[first + i];
      out = d;
    } else {
      float* d = reinterpret_cast<float*>(dyn + a.co.smem_off);
      for (int i = threadIdx.x; i < 6 * n; i += blockDim.x) d[i] = a.co.inv32[first + i];
      out = d;
    }
  }
  __syncthreads();
  return out;
}

// P_i c: translation plus rotation theta x (x_i - centre) / rho of node i's aggregate
__device__ inline d3 coarse_prolong(const PcgArgs& a, int agg, int i, const double* c) {
  const double rs = a.co.rot[agg];
  const d3 r = rs * (ld3(a.co.x, i) - ld3(a.co.centre, agg));
  d3 o = mk(c[0], c[1], c[2]);
  if (rs != 0.0) o = o + mk(c[4] * r.z - c[5] * r.y, c[5] * r.x - c[3] * r.z, c[3] * r.y - c[4] * r.x);
  return o;
}

// End of a solve: CTA 0 reports the iterations, worst status, restarts and
// largest relative residual over the scenes (and every scene's residual and
// iterations when asked).  Status ranks: 0 converged < 3 budget spent <
// 1 breakdown < 2 non-finite.  Every thread of every CTA must call it.
__device__ inline void report_solve(const PcgArgs& a, Shared& sh, bool decider, int sc, int it, int status,
                                    int restarts, double res) {
  if (blockIdx.x != 0) return;
  if (threadIdx.x < 4) sh.agg[threadIdx.x] = 0ull;
  __syncthreads();
  if (decider) {
    const int rank = status == 0 ? 0 : status == 3 ? 1 : status == 1 ? 2 : 3;
    atomicMax(&sh.agg[0], (unsigned long long)it);
    atomicMax(&sh.agg[1], (unsigned long long)rank);
    atomicMax(&sh.agg[2], (unsigned long long)restarts);
    atomicMax(&sh.agg[3], (unsigned long long)__double_as_longlong(fmax(res, 0.0)));
    if (a.sc_res) a.sc_res[sc] = res;
    if (a.sc_it) a.sc_it[sc] = it;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int rank = (int)sh.agg[1];
    a.out[0] = (int)sh.agg[0];
    a.out[1] = rank == 0 ? 0 : rank == 1 ? 3 : rank == 2 ? 1 : 2;
    a.out[2] = (int)sh.agg[2];
    a.res[0] = __longlong_as_double((long long)sh.agg[3]);
  }
}

// ---------------------------------------------------------------------------
// Row products y = A v of the rows a CTA owns, left in shared memory.
// ---------------------------------------------------------------------------
// FEM segment [r0, r1): acc[3 (i - r0) + c].  The contact incidences of the
// segment (a contiguous range of the owner-ordered incidence list) are spread
// over all threads, one chunk of blockDim at a time; within a chunk the
// pieces of one owner's run (split at warp boundaries) are added in thread
// order by the thread holding its last piece, so that every sum is formed in
// the same order in every run.  The BSR part of a row is formed by a group of
// ROWG threads.  Every thread must call it.
template <typename M, typename V, typename A, int ROWG>
__device__ inline void fem_products(const PcgArgs& a, int r0, int r1, int k0, OpView<M> op, const int* colp,
                                    const int* rowp /* relative to k0, indexed from r0; null: global row */,
                                    const M* pairH, const M* fHu, const V* v, A* acc, Shared& sh) {
  // chunk scratch: per-thread run-end pieces (3 values) and the owner of every thread's incidence
  A (*piece)[PCG_THREADS_MAX] = reinterpret_cast<A (*)[PCG_THREADS_MAX]>(&sh.vals[0][0]);
  int* owner_of_t = reinterpret_cast<int*>(&sh.vals[3][0]);
  for (int j = threadIdx.x; j < 3 * (r1 - r0); j += blockDim.x) acc[j] = A(0);
  __syncthreads();
  // incidences e of the segment, consecutive per lane; their owners are non-decreasing, so the
  // contributions of one owner are summed by a segmented warp scan and added once per run
  const int e0 = a.inc_ptr[r0], e1 = (int)min((long long)a.inc_ptr[r1], a.inc_cap);
  const int lane = threadIdx.x & 31;
  for (int eb = e0; eb < e1; eb += blockDim.x) {
    const int e = eb + threadIdx.x;
    int own = -1;
    A y0 = A(0), y1 = A(0), y2 = A(0);
    if (e < e1 && pcg_ok(a, e >= 0 && e < a.inc_cap, 2)) {
      const int2 ie = a.inc[e];
      if (pcg_ok(a, ie.y >= r0 && ie.y < r1, 12)) {
        own = ie.y;
        contact_rows<M, V, A>(a, pairH, fHu, v, ie.x, y0, y1, y2);
      }
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const A t0 = __shfl_up_sync(0xffffffffu, y0, o), t1 = __shfl_up_sync(0xffffffffu, y1, o),
              t2 = __shfl_up_sync(0xffffffffu, y2, o);
      const int ow = __shfl_up_sync(0xffffffffu, own, o);
      if (lane >= o && ow == own) { y0 += t0; y1 += t1; y2 += t2; }
    }
    const int next = __shfl_down_sync(0xffffffffu, own, 1);
    const bool end = own >= 0 && (lane == 31 || next != own);
    piece[0][threadIdx.x] = y0;
    piece[1][threadIdx.x] = y1;
    piece[2][threadIdx.x] = y2;
    owner_of_t[threadIdx.x] = own;
    __syncthreads();
    // the owner's last piece in this chunk: its run does not continue at the next thread
    if (end && !(threadIdx.x + 1 < blockDim.x && owner_of_t[threadIdx.x + 1] == own)) {
      int t0 = threadIdx.x;
      while (t0 > 0 && owner_of_t[t0 - 1] == own) --t0;
      A s0 = A(0), s1 = A(0), s2 = A(0);
      for (int t = t0 | 31; t < (int)threadIdx.x; t += 32) {  // earlier pieces end at lane 31 of their warps
        s0 += piece[0][t]; s1 += piece[1][t]; s2 += piece[2][t];
      }
      s0 += y0; s1 += y1; s2 += y2;
      A* t = acc + 3 * (own - r0);
      t[0] += s0; t[1] += s1; t[2] += s2;
    }
    __syncthreads();
  }
  const int groups = blockDim.x / ROWG, g = threadIdx.x / ROWG, gl = threadIdx.x & (ROWG - 1);
  for (int base = r0; base < r1; base += groups) {
    const int i = base + g;
    A y0 = A(0), y1 = A(0), y2 = A(0);
    if (i < r1) {
      int kb, ke;
      if (rowp) { kb = rowp[i - r0]; ke = rowp[i - r0 + 1]; }
      else { kb = a.row[i] - k0; ke = a.row[i + 1] - k0; }
#pragma unroll 2
      for (int kk = kb + gl; kk < ke; kk += ROWG) {
        const int j = colp[kk];
        if (!pcg_ok(a, j >= 0 && j < a.n_nodes, 1)) continue;
        const A v0 = (A)v[3 * j], v1 = (A)v[3 * j + 1], v2 = (A)v[3 * j + 2];
        const M* H = op.base + (size_t)kk * op.sk;
        const int sq = op.sq;
        y0 = fma((A)H[0], v0, fma((A)H[sq], v1, fma((A)H[2 * sq], v2, y0)));
        y1 = fma((A)H[3 * sq], v0, fma((A)H[4 * sq], v1, fma((A)H[5 * sq], v2, y1)));
        y2 = fma((A)H[6 * sq], v0, fma((A)H[7 * sq], v1, fma((A)H[8 * sq], v2, y2)));
      }
    }
#pragma unroll
    for (int o = ROWG / 2; o > 0; o >>= 1) {
      y0 += __shfl_down_sync(0xffffffffu, y0, o, ROWG);
      y1 += __shfl_down_sync(0xffffffffu, y1, o, ROWG);
      y2 += __shfl_down_sync(0xffffffffu, y2, o, ROWG);
    }
    if (i < r1 && gl == 0) {
      A* c = acc + 3 * (i - r0);
      c[0] += y0; c[1] += y1; c[2] += y2;
    }
  }
  __syncthreads();
}

// The four pseudo-nodes of ABD body b: y into out12[3 t + c].  Thread tid
// serves row t = tid mod 4 (BSR blocks of that row and coupling entries of
// that row, strided by blockDim / 4), then lanes of equal t combine by three
// shuffle levels and warps through shared memory.  Every thread must call it.
template <typename M, typename V, typename A, typename L>
__device__ inline void abd_products(const PcgArgs& a, int b, OpView<M> op, const int* colp, int nloc, const V* v,
                                    const L* list_val, Shared& sh, A* out12) {
  const DevScene& S = a.S;
  const int r = S.nf + 4 * b, k0 = a.row[r];
  const int t = threadIdx.x & 3, slot = threadIdx.x >> 2, nslot = blockDim.x >> 2;
  A y0 = A(0), y1 = A(0), y2 = A(0);
  const int kb = a.row[r + t] - k0, ke = a.row[r + t + 1] - k0;
  for (int kk = kb + slot; kk < ke; kk += nslot) {
    const int j = colp[kk];
    if (!pcg_ok(a, j >= 0 && j < a.n_nodes, 8)) continue;
    const A v0 = (A)v[3 * j], v1 = (A)v[3 * j + 1], v2 = (A)v[3 * j + 2];
    const M* H = op.base + (size_t)kk * op.sk;
    const int sq = op.sq;
    y0 = fma((A)H[0], v0, fma((A)H[sq], v1, fma((A)H[2 * sq], v2, y0)));
    y1 = fma((A)H[3 * sq], v0, fma((A)H[4 * sq], v1, fma((A)H[5 * sq], v2, y1)));
    y2 = fma((A)H[6 * sq], v0, fma((A)H[7 * sq], v1, fma((A)H[8 * sq], v2, y2)));
  }
  // an overflowed list (the Newton iteration is then redone with a larger one) is read only up to its capacity
  const int e0 = a.abd_ptr[b], e1 = (int)min((long long)a.abd_ptr[b + 1], a.abd_cap);
#pragma unroll 4
  for (int e = e0 + 4 * slot + t; e < e1; e += 4 * nslot) {
    if (!pcg_ok(a, e >= 0 && e < a.abd_cap, 9)) break;
    const int code = a.abd_ent[e], j = code >> 2;
    if (!pcg_ok(a, j >= 0 && j < a.n_nodes && (code & 3) == t, 10)) continue;
    const A v0 = (A)v[3 * j], v1 = (A)v[3 * j + 1], v2 = (A)v[3 * j + 2];
    const L* B = list_val + 9 * (size_t)e;
    y0 = fma((A)B[0], v0, fma((A)B[1], v1, fma((A)B[2], v2, y0)));
    y1 = fma((A)B[3], v0, fma((A)B[4], v1, fma((A)B[5], v2, y1)));
    y2 = fma((A)B[6], v0, fma((A)B[7], v1, fma((A)B[8], v2, y2)));
  }
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) {
    y0 += __shfl_xor_sync(0xffffffffu, y0, o);
    y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    y2 += __shfl_xor_sync(0xffffffffu, y2, o);
  }
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane < 4) { sh.red[wi][3 * lane] = y0; sh.red[wi][3 * lane + 1] = y1; sh.red[wi][3 * lane + 2] = y2; }
  __syncthreads();
  if (threadIdx.x < 12) {
    A sum = A(0);
    for (int w = 0; w < nw; ++w) sum += (A)sh.red[w][threadIdx.x];
    out12[threadIdx.x] = sum;
  }
  __syncthreads();
}

// z = D v for one node's 3x3 block (D stored as M, arithmetic in A)
template <typename M, typename A>
__device__ inline void apply3(const M* D, A v0, A v1, A v2, A& z0, A& z1, A& z2) {
  z0 = fma((A)D[0], v0, fma((A)D[1], v1, (A)D[2] * v2));
  z1 = fma((A)D[3], v0, fma((A)D[4], v1, (A)D[5] * v2));
  z2 = fma((A)D[6], v0, fma((A)D[7], v1, (A)D[8] * v2));
}

// One solve (or one per scene of a batch).  M = double: every operation in
// FP64.  M = float: the operator, the contact blocks and the preconditioner
// are stored in FP32 and applied in FP64 arithmetic, so the recurrences see
// one fixed linear operator; the vectors, scalars and dot products are FP64,
// and the FP64 residual b - A x with the FP64 operator is formed whenever the
// recurrence has converged or stagnates, restarting the iteration on it.
//
// Several scenes: each CTA serves the rows of one scene; thread s of every CTA
// runs the scalar recurrences of scene s on that scene's totals (so every CTA
// knows every scene's next action), a scene that has met its tolerance stops
// forming products, and the grid barriers stay common: a loop with a refresh
// anywhere takes the refresh barriers everywhere.
template <typename M, int ROWG>
__global__ void __launch_bounds__(256, 2) k_pcg(PcgArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ Shared sh;
  const DevScene& S = a.S;
  const int nblk = gridDim.x, cta = blockIdx.x;
  const bool fem_cta = cta < a.n_fem_ctas;
  const int nf = S.nf;
  const int n3 = 3 * a.n_nodes;
  const int my_sc = a.cta_scene[cta];
  const bool decider = (int)threadIdx.x < a.n_psc;  // runs the recurrences of scene threadIdx.x
  const int dsc = threadIdx.x;

  // ---- this CTA's rows; shared memory: row products (FEM: 3 per row, ABD: 12
  //      per owned body), then (resident) operator planes, preconditioner, columns, row offsets
  int r0 = 0, r1 = 0, k0 = 0, nloc = 0, ab0 = 0, ab1 = 0;
  OpView<M> op{nullptr, 0, 1};
  const int* colp = nullptr;
  const int* rowp = nullptr;
  const M* dinv_loc = nullptr;
  const M* opM = (const M*)a.op;
  const M* dinvM = (const M*)a.dinv;
  double* acc = (double*)dyn;
  if (fem_cta) {
    r0 = a.seg_row[cta]; r1 = a.seg_row[cta + 1];
    if (!pcg_ok(a, r0 >= 0 && r0 <= r1 && r1 <= nf, 11)) r0 = r1 = 0;
    k0 = a.row[r0]; nloc = a.row[r1] - k0;
    if (a.resident) {
      M* s_op = (M*)(acc + a.acc_doubles);
      M* s_dinv = s_op + 9 * (size_t)nloc;
      int* s_col = (int*)(s_dinv + 9 * (size_t)(r1 - r0));
      int* s_row = s_col + nloc;
      const M* g_op = opM + 9 * (size_t)k0;
      for (int idx = threadIdx.x; idx < 9 * nloc; idx += blockDim.x) s_op[idx] = g_op[idx];
      for (int idx = threadIdx.x; idx < 9 * (r1 - r0); idx += blockDim.x) s_dinv[idx] = dinvM[9 * (size_t)r0 + idx];
      for (int idx = threadIdx.x; idx < nloc; idx += blockDim.x) s_col[idx] = a.col[k0 + idx];
      for (int idx = threadIdx.x; idx <= r1 - r0; idx += blockDim.x) s_row[idx] = a.row[r0 + idx] - k0;
      __syncthreads();
      op = OpView<M>{s_op, nloc, 1};
      colp = s_col; rowp = s_row; dinv_loc = s_dinv;
    } else {
      op = OpView<M>{opM + 9 * (size_t)k0, nloc, 1};
      colp = a.col + k0; dinv_loc = dinvM + 9 * (size_t)r0;
    }
  } else {
    ab0 = a.abd_seg[cta - a.n_fem_ctas]; ab1 = a.abd_seg[cta - a.n_fem_ctas + 1];
    if (!pcg_ok(a, ab0 >= 0 && ab0 <= ab1 && ab1 <= S.nab, 13)) ab0 = ab1 = 0;
  }
  // preconditioner block of node i (owned by this CTA)
  auto Dof = [&](int i) -> const M* { return (fem_cta ? dinv_loc + 9 * (size_t)(i - r0) : dinvM + 9 * (size_t)i); };
  // threads that own a node in the first pass of for_nodes (the others hold zero partial sums)
  const int n_act = fem_cta ? r1 - r0 : 4;
  // coarse level: this CTA's aggregate (its FEM rows), -1 without one; the coarse images of w and z of
  // the CTA's aggregate, identical in every thread
  const bool coarse = a.co.inv32 != nullptr;
  const int my_agg = (coarse && fem_cta && my_sc >= 0 && r1 > r0) ? a.co.cta_agg[cta] : -1;
  const void* co_rows = coarse_stage(a, my_agg, my_sc, dyn);
  double co_w[6] = {0, 0, 0, 0, 0, 0}, co_z[6] = {0, 0, 0, 0, 0, 0};

  Vecs<double> V;
  {
    double* base = (double*)a.vec;
    V.r = base; V.u = base + n3; V.w = base + 2 * (size_t)n3; V.m0 = base + 3 * (size_t)n3;
    V.m1 = base + 4 * (size_t)n3; V.z = base + 5 * (size_t)n3; V.q = base + 6 * (size_t)n3;
    V.s = base + 7 * (size_t)n3; V.p = base + 8 * (size_t)n3;
  }
  const M* pairH = (const M*)a.pairH;
  const M* fHu = (const M*)a.fHu;
  double* x = a.x;
  double* t64 = a.t64;
  // partial sums: [R][2 parities][3][grid], then the residual norms [R][grid]
  double* partT = (double*)a.partial;
  const size_t repT = 2 * 3 * (size_t)nblk;
  double* partD = partT + PCG_REPLICAS * repT;
  const int myrep = cta % PCG_REPLICAS;

  // y = A v for every owned row, left in shared memory: the iteration
  // operator (assembled = false: layout copy of type M) or the assembled FP64
  // one.  Every thread of the CTA must call it.
  auto products = [&](bool assembled, auto&& op_view_fem, const int* colp_fem, const int* rowp_fem, auto mtag,
                      const auto* mat_pairH, const auto* mat_fHu, const double* vin) {
    using MM = decltype(mtag);
    if (fem_cta) {
      fem_products<MM, double, double, ROWG>(a, r0, r1, k0, op_view_fem, colp_fem, rowp_fem, mat_pairH, mat_fHu,
                                             vin, acc, sh);
    } else {
      for (int b = ab0, j = 0; b < ab1; ++b, ++j) {
        const int rr = nf + 4 * b, kb0 = a.row[rr], nl = a.row[rr + 4] - kb0;
        OpView<MM> ov = assembled ? OpView<MM>{(const MM*)a.val64 + 9 * (size_t)kb0, 1, 9}
                                  : OpView<MM>{(const MM*)a.op + 9 * (size_t)kb0, nl, 1};
        abd_products<MM, double, double, double>(a, b, ov, a.col + kb0, nl, vin, a.abd_val, sh, acc + 12 * j);
      }
    }
  };
  // node-local pass over the owned nodes, with the node's row product from `products`
  auto for_nodes = [&](auto&& fn) {
    if (fem_cta) {
      for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) fn(i, acc + 3 * (i - r0));
    } else {
      for (int b = ab0, j = 0; b < ab1; ++b, ++j)
        if (threadIdx.x < 4) fn(nf + 4 * b + threadIdx.x, acc + 12 * j + 3 * threadIdx.x);
    }
  };
  // this CTA's part of a norm, to partD (every replica)
  auto write_norm = [&](double v) {
    double w[1] = {v};
    cta_sum<1, double>(w, sh);
    if (threadIdx.x < PCG_REPLICAS) partD[threadIdx.x * (size_t)nblk + cta] = sh.out[0];
    __syncthreads();
  };
  // the FP64 operator (assembled layout) for the true residual
  OpView<double> op64{a.val64 + 9 * (size_t)k0, 1, 9};
  const int* col64 = a.col + k0;

  // ---- x = 0, t64 = b, |b|^2 of every scene
  {
    double v = 0.0;
    for_nodes([&](int i, const double*) {
      for (int c = 0; c < 3; ++c) {
        double bv = a.b[3 * i + c];
        x[3 * i + c] = 0.0;
        t64[3 * i + c] = bv;
        v += bv * bv;
      }
    });
    write_norm(v);
  }
  grid.sync();
  scene_totals<1, double>(a, partD + myrep * (size_t)nblk, nblk, sh, nullptr);

  // ---- per-scene state, held by the scene's decision thread
  constexpr bool F32 = sizeof(M) == 4;
  constexpr int STALL = 80;  // iterations without a new minimum of the recursive residual before a refresh
  const int max_replace = a.max_replace > 0 ? a.max_replace : 10;
  double bb = 0.0, tol2_true = 0.0, sigma = 1.0, unscale = 1.0, tt = 0.0, tol_in2 = 0.0;
  double alpha_old = 1.0, gamma_old = 1.0, rr_best = 0.0;
  int it = 0, it_best = 0, replaced = 0, status = 0;
  bool fresh = true, done = true;
  // inner target in the scaled units of the current restart: the requested
  // reduction, but not below what the FP32-stored operator resolves
  auto inner_tol2 = [&]() -> double {
    double t = tol2_true * sigma * sigma;
    if (F32) t = fmax(t, 1e-12);
    return t;
  };
  if (decider) {
    bb = scene_total(a, sh, 0, dsc);
    const bool skip = a.scene_skip && a.scene_skip[dsc];
    done = skip || !(bb > 0.0) || !isfinite(bb);
    status = (skip || isfinite(bb)) ? 0 : 2;
    if (skip) bb = 0.0;
    tt = bb;
    tol2_true = a.rtol * a.rtol * bb;
    unscale = sqrt(bb);
    sigma = done ? 1.0 : 1.0 / unscale;
    tol_in2 = inner_tol2();
    if (dsc == my_sc) { sh.action = done ? 0 : 1; sh.scal[3] = sigma; }
  }
  __syncthreads();
  bool my_run = my_sc >= 0 && sh.action;  // this CTA's scene forms products in the next loop
  __syncthreads();

  // ---- (re)start of the scenes whose CTAs have on = true, from t64 = b - A x:
  //      r = sigma t64, u = M^-1 r, w = A u, m = M^-1 w, partial sums into parity par.
  //      Two grid barriers, taken by every CTA.
  auto restart = [&](int par, bool on) {
    if (on) {
      const double sg = sh.scal[3];
      for_nodes([&](int i, const double*) {
        for (int c = 0; c < 3; ++c) {
          const int q = 3 * i + c;
          V.r[q] = sg * t64[q];
          V.z[q] = 0.0; V.q[q] = 0.0; V.s[q] = 0.0; V.p[q] = 0.0;
        }
      });
    }
    // coarse image of r (its restriction must be complete before any CTA applies the inverse)
    double cr[6] = {0, 0, 0, 0, 0, 0};
    if (coarse) {
      __syncthreads();
      if (on) coarse_restrict(a, my_agg, r0, r1, sh, [&](int i, double& v0, double& v1, double& v2) {
        v0 = V.r[3 * i]; v1 = V.r[3 * i + 1]; v2 = V.r[3 * i + 2];
      });
      grid.sync();
      if (on) coarse_own(a, my_agg, my_sc, sh, cr, co_rows);
    }
    if (on) {
      for_nodes([&](int i, const double*) {
        const int q = 3 * i;
        double u0, u1, u2;
        apply3<M, double>(Dof(i), V.r[q], V.r[q + 1], V.r[q + 2], u0, u1, u2);
        if (my_agg >= 0) {
          const d3 cc = coarse_prolong(a, my_agg, i, cr);
          u0 += cc.x; u1 += cc.y; u2 += cc.z;
        }
        V.u[q] = u0; V.u[q + 1] = u1; V.u[q + 2] = u2;
      });
    }
    grid.sync();
    if (on) products(false, op, colp, rowp, M(0), pairH, fHu, V.u);
    double cwv[6] = {0, 0, 0, 0, 0, 0};
    if (coarse) {
      // coarse image of w = A u: c_w = A_c^-1 P^T w, c_z = 0
      if (on) coarse_restrict(a, my_agg, r0, r1, sh, [&](int i, double& v0, double& v1, double& v2) {
        const double* y = acc + 3 * (i - r0);
        v0 = y[0]; v1 = y[1]; v2 = y[2];
      });
      grid.sync();
      if (on) coarse_own(a, my_agg, my_sc, sh, cwv, co_rows);
      if (on)
        for (int k = 0; k < 6; ++k) { co_w[k] = cwv[k]; co_z[k] = 0.0; }
    }
    if (on) {
      double* mdst = par ? V.m1 : V.m0;
      double pv[3] = {0.0, 0.0, 0.0};
      for_nodes([&](int i, const double* y) {
        const int q = 3 * i;
        V.w[q] = y[0]; V.w[q + 1] = y[1]; V.w[q + 2] = y[2];
        double m0, m1, m2;
        apply3<M, double>(Dof(i), y[0], y[1], y[2], m0, m1, m2);
        if (my_agg >= 0) {
          const d3 cc = coarse_prolong(a, my_agg, i, cwv);
          m0 += cc.x; m1 += cc.y; m2 += cc.z;
        }
        mdst[q] = m0; mdst[q + 1] = m1; mdst[q + 2] = m2;
        const double u0 = V.u[q], u1 = V.u[q + 1], u2 = V.u[q + 2];
        const double rr0 = V.r[q], rr1 = V.r[q + 1], rr2 = V.r[q + 2];
        pv[0] += rr0 * u0 + rr1 * u1 + rr2 * u2;
        pv[1] += y[0] * u0 + y[1] * u1 + y[2] * u2;
        pv[2] += rr0 * rr0 + rr1 * rr1 + rr2 * rr2;
      });
      write_partials<double>(partT + (size_t)par * 3 * nblk, repT, nblk, sh, pv, n_act);
    }
    grid.sync();
  };
  restart(0, my_run);

  enum { ACT_IDLE = 0, ACT_STEP = 1, ACT_REFRESH = 2 };
  for (int L = 0;; ++L) {
    const int par = L & 1;
    const double* rep = partT + (size_t)par * 3 * nblk + myrep * repT;
    double* mcur = par ? V.m1 : V.m0;
    double* mnext = par ? V.m0 : V.m1;
    // one solve: the partial sums are loaded first, the product n = A m is formed while they arrive
    Partials<double> P;
    if (a.n_psc == 1) load_partials<double>(rep, nblk, P);
    if (my_run) products(false, op, colp, rowp, M(0), pairH, fHu, mcur);
    // coarse restriction of n = A m (read by every CTA of the solve after the coarse barrier below)
    if (coarse && my_run)
      coarse_restrict(a, my_agg, r0, r1, sh, [&](int i, double& v0, double& v1, double& v2) {
        const double* y = acc + 3 * (i - r0);
        v0 = y[0]; v1 = y[1]; v2 = y[2];
      });
    scene_totals<3, double>(a, rep, nblk, sh, a.n_psc == 1 ? &P : nullptr);
    // the scalar recurrences of every scene (identical inputs in every CTA, identical results); the
    // CTA's own scene reaches its threads through shared memory
    int act = ACT_IDLE;
    if (decider && !done) {
      const double gamma = scene_total(a, sh, 0, dsc), delta = scene_total(a, sh, 1, dsc),
                   rr = scene_total(a, sh, 2, dsc);
      double al = 0.0, be = 0.0;
      act = ACT_STEP;
      if (!isfinite(rr) || !isfinite(delta) || !isfinite(gamma)) { status = 2; done = true; act = ACT_IDLE; }
      else {
        if (fresh || rr < rr_best) { rr_best = rr; it_best = it; }
        if (rr <= tol_in2 || it - it_best > STALL || it >= a.max_iter) act = ACT_REFRESH;
        else if (!(gamma > 0.0)) {
          // r^T M^-1 r <= 0 with r != 0: the preconditioner is not positive definite (breakdown)
          status = 1; done = true; act = ACT_IDLE;
        } else if (fresh) {
          if (!(delta > 0.0)) { status = 1; done = true; act = ACT_IDLE; }
          else al = gamma / delta;
        } else {
          be = gamma / gamma_old;
          const double den = delta - be * gamma / alpha_old;
          if (!(den > 0.0)) act = ACT_REFRESH;  // lost conjugacy: refresh from the true residual
          else al = gamma / den;
        }
      }
      if (act == ACT_STEP) {
        gamma_old = gamma;
        alpha_old = al;
        fresh = false;
        ++it;
      }
      if (dsc == my_sc) {
        sh.scal[0] = al;
        sh.scal[1] = be;
        sh.scal[2] = al * unscale;
      }
    }
    if (decider && dsc == my_sc) sh.action = act;
    const bool any_refresh = __syncthreads_or(act == ACT_REFRESH);
    const bool any_live = __syncthreads_or(act != ACT_IDLE);
    const int my_act = my_sc >= 0 ? sh.action : ACT_IDLE;
    const double alpha = sh.scal[0], beta = sh.scal[1], ax = sh.scal[2];
    if (!any_live) break;
    // coarse images: c_z = A_c^-1 P^T n + beta c_z, c_w = c_w - alpha c_z (the recurrences of z and w)
    double cwv[6] = {0, 0, 0, 0, 0, 0};
    if (coarse) {
      grid.sync();
      if (my_act == ACT_STEP) {
        double eta[6];
        coarse_own(a, my_agg, my_sc, sh, eta, co_rows);
        for (int k = 0; k < 6; ++k) {
          co_z[k] = fma(beta, co_z[k], eta[k]);
          co_w[k] = fma(-alpha, co_z[k], co_w[k]);
          cwv[k] = co_w[k];
        }
      }
    }
    if (my_act == ACT_STEP) {
      // every recurrence of the owned nodes, one thread per node
      double pv[3] = {0.0, 0.0, 0.0};
      for_nodes([&](int i, const double* n) {
        // every value of the node is loaded before anything is stored (the vectors may alias as far as
        // the compiler knows, which would otherwise serialise the loads behind the stores)
        double oz[3], oq[3], os[3], op_[3], ou[3], ow[3], orr[3], om[3], ox[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int q = 3 * i + c;
          oz[c] = V.z[q]; oq[c] = V.q[q]; os[c] = V.s[q]; op_[c] = V.p[q]; ou[c] = V.u[q];
          ow[c] = V.w[q]; orr[c] = V.r[q]; om[c] = mcur[q]; ox[c] = x[q];
        }
        double rn[3], un[3], wn[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int q = 3 * i + c;
          const double z = fma(beta, oz[c], n[c]);
          const double qq = fma(beta, oq[c], om[c]);
          const double s = fma(beta, os[c], ow[c]);
          const double p = fma(beta, op_[c], ou[c]);
          V.z[q] = z; V.q[q] = qq; V.s[q] = s; V.p[q] = p;
          x[q] = fma(ax, p, ox[c]);
          rn[c] = fma(-alpha, s, orr[c]);
          un[c] = fma(-alpha, qq, ou[c]);
          wn[c] = fma(-alpha, z, ow[c]);
          V.r[q] = rn[c]; V.u[q] = un[c]; V.w[q] = wn[c];
        }
        double m0, m1, m2;
        apply3<M, double>(Dof(i), wn[0], wn[1], wn[2], m0, m1, m2);
        if (my_agg >= 0) {
          const d3 cc = coarse_prolong(a, my_agg, i, cwv);
          m0 += cc.x; m1 += cc.y; m2 += cc.z;
        }
        mnext[3 * i] = m0; mnext[3 * i + 1] = m1; mnext[3 * i + 2] = m2;
        pv[0] += rn[0] * un[0] + rn[1] * un[1] + rn[2] * un[2];
        pv[1] += wn[0] * un[0] + wn[1] * un[1] + wn[2] * un[2];
        pv[2] += rn[0] * rn[0] + rn[1] * rn[1] + rn[2] * rn[2];
      });
      write_partials<double>(partT + (size_t)(par ^ 1) * 3 * nblk, repT, nblk, sh, pv, n_act);
    }
    bool my_restart = false;
    if (any_refresh) {
      // ---- the FP64 residual t64 = b - A64 x of the refreshing scenes (their x is unchanged in this loop)
      const bool ref = my_act == ACT_REFRESH;
      if (ref) {
        products(true, op64, col64, (const int*)nullptr, 0.0, a.pairH64, a.fHu64, x);
        double v = 0.0;
        for_nodes([&](int i, const double* y) {
          const int q = 3 * i;
          const double t0 = a.b[q] - y[0], t1 = a.b[q + 1] - y[1], t2 = a.b[q + 2] - y[2];
          t64[q] = t0; t64[q + 1] = t1; t64[q + 2] = t2;
          v += t0 * t0 + t1 * t1 + t2 * t2;
        });
        write_norm(v);
      }
      grid.sync();
      scene_totals<1, double>(a, partD + myrep * (size_t)nblk, nblk, sh, nullptr);
      if (act == ACT_REFRESH) {  // decision threads of the refreshing scenes
        tt = scene_total(a, sh, 0, dsc);
        bool again = false;
        if (!isfinite(tt)) { status = 2; done = true; }
        else if (tt <= tol2_true || it >= a.max_iter || replaced >= max_replace) done = true;
        else {
          ++replaced;
          unscale = sqrt(tt);
          sigma = 1.0 / unscale;
          tol_in2 = inner_tol2();
          fresh = true;
          again = true;
        }
        if (dsc == my_sc) { sh.action = again ? 1 : 0; sh.scal[3] = sigma; }
      }
      __syncthreads();
      my_restart = ref && sh.action;
      __syncthreads();
      restart(par ^ 1, my_restart);
    } else {
      grid.sync();
    }
    my_run = my_act == ACT_STEP || my_restart;
  }
  if (decider && status == 0 && !(tt <= tol2_true)) status = 3;  // budget spent before the tolerance
  report_solve(a, sh, decider, dsc, it, status, replaced, decider && bb > 0.0 ? sqrt(fmax(tt, 0.0) / bb) : 0.0);
}

// Mixed-precision solve: iterative refinement around an FP32 conjugate-
// gradient solve.  The inner solve runs entirely in FP32 (operator,
// preconditioner, contact blocks, vectors, dot products) in the
// Chronopoulos-Gear form of CG, which tolerates the rounding of FP32 matrix
// products (the pipelined recurrences do not): two grid barriers per
// iteration, one reduction point.  Its solution d of A32 d = sigma (b - A x)
// is accumulated into x in FP64 and the FP64 residual b - A x is recomputed
// with the FP64 operator until it meets the tolerance.  Several scenes: as in
// k_pcg, every scene has its own recurrences, refinements and stop, and a loop
// in which any scene ends an inner solve takes the refinement barriers
// everywhere.
template <int ROWG>
__global__ void __launch_bounds__(256, 2) k_pcg32(PcgArgs a) {
  using F = float;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ Shared sh;
  const DevScene& S = a.S;
  const int nblk = gridDim.x, cta = blockIdx.x;
  const bool fem_cta = cta < a.n_fem_ctas;
  const int nf = S.nf;
  const int n3 = 3 * a.n_nodes;
  const int my_sc = a.cta_scene[cta];
  const bool decider = (int)threadIdx.x < a.n_psc;  // runs the recurrences of scene threadIdx.x
  const int dsc = threadIdx.x;

  int r0 = 0, r1 = 0, k0 = 0, nloc = 0, ab0 = 0, ab1 = 0;
  OpView<F> op{nullptr, 0, 1};
  const int* colp = nullptr;
  const int* rowp = nullptr;
  const F* dinv_loc = nullptr;
  const F* opF = (const F*)a.op;
  const F* dinvF = (const F*)a.dinv;
  double* acc = (double*)dyn;  // row products: FP64 for the residual, FP32 for the iteration
  F* accf = (F*)dyn;
  if (fem_cta) {
    r0 = a.seg_row[cta]; r1 = a.seg_row[cta + 1];
    if (!pcg_ok(a, r0 >= 0 && r0 <= r1 && r1 <= nf, 11)) r0 = r1 = 0;
    k0 = a.row[r0]; nloc = a.row[r1] - k0;
    if (a.resident) {
      F* s_op = (F*)(acc + a.acc_doubles);
      F* s_dinv = s_op + 9 * (size_t)nloc;
      int* s_col = (int*)(s_dinv + 9 * (size_t)(r1 - r0));
      int* s_row = s_col + nloc;
      const F* g_op = opF + 9 * (size_t)k0;
      for (int idx = threadIdx.x; idx < 9 * nloc; idx += blockDim.x) s_op[idx] = g_op[idx];
      for (int idx = threadIdx.x; idx < 9 * (r1 - r0); idx += blockDim.x) s_dinv[idx] = dinvF[9 * (size_t)r0 + idx];
      for (int idx = threadIdx.x; idx < nloc; idx += blockDim.x) s_col[idx] = a.col[k0 + idx];
      for (int idx = threadIdx.x; idx <= r1 - r0; idx += blockDim.x) s_row[idx] = a.row[r0 + idx] - k0;
      __syncthreads();
      op = OpView<F>{s_op, nloc, 1};
      colp = s_col; rowp = s_row; dinv_loc = s_dinv;
    } else {
      op = OpView<F>{opF + 9 * (size_t)k0, nloc, 1};
      colp = a.col + k0; dinv_loc = dinvF + 9 * (size_t)r0;
    }
  } else {
    ab0 = a.abd_seg[cta - a.n_fem_ctas]; ab1 = a.abd_seg[cta - a.n_fem_ctas + 1];
    if (!pcg_ok(a, ab0 >= 0 && ab0 <= ab1 && ab1 <= S.nab, 13)) ab0 = ab1 = 0;
  }
  auto Dof = [&](int i) -> const F* { return (fem_cta ? dinv_loc + 9 * (size_t)(i - r0) : dinvF + 9 * (size_t)i); };
  // coarse level: this CTA's aggregate (its FEM rows), -1 without one, applied in FP32; the coarse
  // images of r and s of the CTA's aggregate, identical in every thread
  const bool coarse = a.co.inv32 != nullptr;
  const int my_agg = (coarse && fem_cta && my_sc >= 0 && r1 > r0) ? a.co.cta_agg[cta] : -1;
  const void* co_rows = coarse_stage(a, my_agg, my_sc, dyn);
  F co_r[6] = {F(0), F(0), F(0), F(0), F(0), F(0)}, co_s[6] = {F(0), F(0), F(0), F(0), F(0), F(0)};

  F* base = (F*)a.vec;
  F* r = base;
  F* u = base + n3;
  F* w = base + 2 * (size_t)n3;
  F* pv_ = base + 3 * (size_t)n3;
  F* sv = base + 4 * (size_t)n3;
  F* xi = base + 5 * (size_t)n3;
  const F* pairH = (const F*)a.pairH;
  const F* fHu = (const F*)a.fHu;
  double* x = a.x;
  double* t64 = a.t64;
  // partial sums: FP32 [R][2][3][grid], then FP64 [R][grid] (norms of b and of the true residual)
  F* partF = (F*)a.partial;
  const size_t repT = 2 * 3 * (size_t)nblk;
  double* partD = (double*)a.partial + PCG_REPLICAS * repT;
  const int myrep = cta % PCG_REPLICAS;

  // FP32 products of the iteration operator, FP64 products of the assembled one
  auto products32 = [&](const F* vin) {
    if (fem_cta) {
      fem_products<F, F, F, ROWG>(a, r0, r1, k0, op, colp, rowp, pairH, fHu, vin, accf, sh);
    } else {
      for (int b = ab0, j = 0; b < ab1; ++b, ++j) {
        const int rr = nf + 4 * b, kb0 = a.row[rr], nl = a.row[rr + 4] - kb0;
        abd_products<F, F, F, F>(a, b, OpView<F>{opF + 9 * (size_t)kb0, nl, 1}, a.col + kb0, nl, vin, a.abd_val32, sh,
                                 accf + 12 * j);
      }
    }
  };
  auto products64 = [&](const double* vin) {
    if (fem_cta) {
      fem_products<double, double, double, ROWG>(a, r0, r1, k0, OpView<double>{a.val64 + 9 * (size_t)k0, 1, 9},
                                                 a.col + k0, nullptr, a.pairH64, a.fHu64, vin, acc, sh);
    } else {
      for (int b = ab0, j = 0; b < ab1; ++b, ++j) {
        const int rr = nf + 4 * b, kb0 = a.row[rr], nl = a.row[rr + 4] - kb0;
        abd_products<double, double, double, double>(a, b, OpView<double>{a.val64 + 9 * (size_t)kb0, 1, 9},
                                                     a.col + kb0, nl, vin, a.abd_val, sh, acc + 12 * j);
      }
    }
  };
  // node-local pass; the row product of the node (from the last products call) is at offset o
  auto for_nodes = [&](auto&& fn) {
    if (fem_cta) {
      for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) fn(i, 3 * (i - r0));
    } else {
      for (int b = ab0, j = 0; b < ab1; ++b, ++j)
        if (threadIdx.x < 4) fn(nf + 4 * b + threadIdx.x, 12 * j + 3 * threadIdx.x);
    }
  };
  auto write_norm = [&](double v) {
    double wv[1] = {v};
    cta_sum<1, double>(wv, sh);
    if (threadIdx.x < PCG_REPLICAS) partD[threadIdx.x * (size_t)nblk + cta] = sh.out[0];
    __syncthreads();
  };

  // ---- x = 0, t64 = b, |b|^2 of every scene
  {
    double v = 0.0;
    for_nodes([&](int i, int) {
      for (int c = 0; c < 3; ++c) {
        const double bv = a.b[3 * i + c];
        x[3 * i + c] = 0.0;
        t64[3 * i + c] = bv;
        v += bv * bv;
      }
    });
    write_norm(v);
  }
  grid.sync();
  scene_totals<1, double>(a, partD + myrep * (size_t)nblk, nblk, sh, nullptr);

  // ---- per-scene state, held by the scene's decision thread
  constexpr int STALL = 80;
  constexpr int MAX_REFINE = 10;
  double bb = 0.0, tol2_true = 0.0, tt = 0.0, unscale = 1.0;
  F tol_in2 = F(0), alpha_old = F(1), gamma_old = F(1), rr_best = F(0);
  int it = 0, it_best = 0, refine = 0, status = 0;
  bool fresh = true, done = true;
  // a new inner solve of A32 d = sigma t64 from d = 0; its target is the
  // remaining reduction, not below what FP32 CG resolves
  auto begin_inner = [&]() {
    unscale = sqrt(tt);
    tol_in2 = (F)fmax(tol2_true / tt, 1e-10);
    fresh = true;
    alpha_old = F(1);
    gamma_old = F(1);
    rr_best = F(0);
    it_best = it;
    if (dsc == my_sc) { sh.scal[2] = unscale; sh.scal[3] = 1.0 / unscale; }
  };
  if (decider) {
    bb = scene_total(a, sh, 0, dsc);
    const bool skip = a.scene_skip && a.scene_skip[dsc];
    done = skip || !(bb > 0.0) || !isfinite(bb);
    status = (skip || isfinite(bb)) ? 0 : 2;
    if (skip) bb = 0.0;
    tt = bb;
    tol2_true = a.rtol * a.rtol * bb;
    if (!done) begin_inner();
    if (dsc == my_sc) sh.action = done ? 0 : 1;
  }
  __syncthreads();
  bool my_run = my_sc >= 0 && sh.action;  // this CTA's scene is inside an inner solve
  __syncthreads();

  // inner solve start of this CTA's scene: r = sigma t64, u = M^-1 r, p = s = d = 0, and the
  // CTA's parts of (r, u), (r, r)
  F g_l = F(0), rr_l = F(0);
  // every CTA must call it (the coarse level takes a grid barrier); `on`: this CTA's scene starts an
  // inner solve
  auto init_inner = [&](bool on) {
    const double sigma = sh.scal[3];
    if (on) {
      g_l = F(0);
      rr_l = F(0);
    }
    if (on)
      for_nodes([&](int i, int) {
        for (int c = 0; c < 3; ++c) {
          const int q = 3 * i + c;
          r[q] = (F)(sigma * t64[q]);
          pv_[q] = F(0); sv[q] = F(0); xi[q] = F(0);
        }
      });
    // coarse image of r: c_r = A_c^-1 P^T r, c_s = 0
    double cr[6] = {0, 0, 0, 0, 0, 0};
    if (coarse) {
      __syncthreads();
      if (on) coarse_restrict(a, my_agg, r0, r1, sh, [&](int i, double& v0, double& v1, double& v2) {
        v0 = r[3 * i]; v1 = r[3 * i + 1]; v2 = r[3 * i + 2];
      });
      grid.sync();
      if (on) {
        coarse_own(a, my_agg, my_sc, sh, cr, co_rows);
        for (int k = 0; k < 6; ++k) { co_r[k] = (F)cr[k]; co_s[k] = F(0); }
      }
    }
    if (on)
      for_nodes([&](int i, int) {
        F rv[3] = {r[3 * i], r[3 * i + 1], r[3 * i + 2]}, uv[3];
        apply3<F, F>(Dof(i), rv[0], rv[1], rv[2], uv[0], uv[1], uv[2]);
        if (my_agg >= 0) {
          const d3 cc = coarse_prolong(a, my_agg, i, cr);
          uv[0] += (F)cc.x; uv[1] += (F)cc.y; uv[2] += (F)cc.z;
        }
        for (int c = 0; c < 3; ++c) u[3 * i + c] = uv[c];
        g_l += rv[0] * uv[0] + rv[1] * uv[1] + rv[2] * uv[2];
        rr_l += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
      });
  };
  init_inner(my_run);
  grid.sync();

  enum { ACT_IDLE = 0, ACT_STEP = 1, ACT_END = 2 };
  for (int L = 0;; ++L) {
    const int par = L & 1;
    // phase A: w = A u, partial sums of (r, u), (w, u), (r, r)
    if (my_run) {
      products32(u);
      F d_l = F(0);
      for_nodes([&](int i, int o) {
        const int q = 3 * i;
        const F w0 = accf[o], w1 = accf[o + 1], w2 = accf[o + 2];
        w[q] = w0; w[q + 1] = w1; w[q + 2] = w2;
        d_l += w0 * u[q] + w1 * u[q + 1] + w2 * u[q + 2];
      });
      const F pl[3] = {g_l, d_l, rr_l};
      write_partials<F>(partF + (size_t)par * 3 * nblk, repT, nblk, sh, pl);
      // coarse restriction of w = A u (read by every CTA of the solve after the barrier)
      if (coarse)
        coarse_restrict(a, my_agg, r0, r1, sh, [&](int i, double& v0, double& v1, double& v2) {
          v0 = w[3 * i]; v1 = w[3 * i + 1]; v2 = w[3 * i + 2];
        });
    }
    grid.sync();
    // phase B: totals, the scalars of every scene, vector updates
    {
      const F* rep = partF + (size_t)par * 3 * nblk + myrep * repT;
      Partials<F> P;
      if (a.n_psc == 1) load_partials<F>(rep, nblk, P);
      scene_totals<3, F>(a, rep, nblk, sh, a.n_psc == 1 ? &P : nullptr);
    }
    int act = ACT_IDLE;
    if (decider && !done) {
      const F gamma = (F)scene_total(a, sh, 0, dsc), delta = (F)scene_total(a, sh, 1, dsc),
              rr = (F)scene_total(a, sh, 2, dsc);
      F al = F(0), be = F(0);
      act = ACT_STEP;
      if (!isfinite(rr) || !isfinite(delta) || !isfinite(gamma)) { status = 2; done = true; act = ACT_IDLE; }
      else {
        if (fresh || rr < rr_best) { rr_best = rr; it_best = it; }
        if (rr <= tol_in2 || it - it_best > STALL || it >= a.max_iter) act = ACT_END;
        else if (!(gamma > F(0))) {
          // r^T M^-1 r <= 0 with r != 0: the preconditioner is not positive definite (breakdown)
          status = 1; done = true; act = ACT_IDLE;
        } else if (fresh) {
          if (!(delta > F(0))) { status = 1; done = true; act = ACT_IDLE; }
          else al = gamma / delta;
        } else {
          be = gamma / gamma_old;
          const F den = delta - be * gamma / alpha_old;
          if (!(den > F(0))) act = ACT_END;  // lost conjugacy: refine from the true residual
          else al = gamma / den;
        }
        gamma_old = gamma;
        alpha_old = al;
      }
      if (act == ACT_STEP) { fresh = false; ++it; }
      if (dsc == my_sc) { sh.scal[0] = al; sh.scal[1] = be; }
    }
    if (decider && dsc == my_sc) sh.action = act;
    const bool any_end = __syncthreads_or(act == ACT_END);
    const bool any_live = __syncthreads_or(act != ACT_IDLE);
    const int my_act = my_sc >= 0 ? sh.action : ACT_IDLE;
    const F alpha = (F)sh.scal[0], beta = (F)sh.scal[1];
    if (!any_live) break;
    // coarse images: c_s = A_c^-1 P^T w + beta c_s, c_r = c_r - alpha c_s (the recurrences of s and r)
    double crv[6] = {0, 0, 0, 0, 0, 0};
    if (coarse && my_act == ACT_STEP) {
      double eta[6];
      coarse_own(a, my_agg, my_sc, sh, eta, co_rows);
      for (int k = 0; k < 6; ++k) {
        co_s[k] = fmaf(beta, co_s[k], (F)eta[k]);
        co_r[k] = fmaf(-alpha, co_s[k], co_r[k]);
        crv[k] = (double)co_r[k];
      }
    }
    if (my_act == ACT_STEP) {
      g_l = F(0);
      rr_l = F(0);
      for_nodes([&](int i, int) {
        F ou[3], opv[3], ow[3], osv[3], oxi[3], orr[3], rn[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int q = 3 * i + c;
          ou[c] = u[q]; opv[c] = pv_[q]; ow[c] = w[q]; osv[c] = sv[q]; oxi[c] = xi[q]; orr[c] = r[q];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int q = 3 * i + c;
          const F p = fmaf(beta, opv[c], ou[c]);
          const F sq = fmaf(beta, osv[c], ow[c]);
          pv_[q] = p;
          sv[q] = sq;
          xi[q] = fmaf(alpha, p, oxi[c]);
          rn[c] = fmaf(-alpha, sq, orr[c]);
          r[q] = rn[c];
        }
        F un[3];
        apply3<F, F>(Dof(i), rn[0], rn[1], rn[2], un[0], un[1], un[2]);
        if (my_agg >= 0) {
          const d3 cc = coarse_prolong(a, my_agg, i, crv);
          un[0] += (F)cc.x; un[1] += (F)cc.y; un[2] += (F)cc.z;
        }
        for (int c = 0; c < 3; ++c) u[3 * i + c] = un[c];
        g_l += rn[0] * un[0] + rn[1] * un[1] + rn[2] * un[2];
        rr_l += rn[0] * rn[0] + rn[1] * rn[1] + rn[2] * rn[2];
      });
    }
    bool my_again = false;
    if (any_end) {
      // ---- scenes that ended an inner solve: x += d / sigma in FP64, then the FP64 residual
      const bool fin = my_act == ACT_END;
      if (fin) {
        const double us = sh.scal[2];
        for_nodes([&](int i, int) {
          for (int c = 0; c < 3; ++c) x[3 * i + c] += us * (double)xi[3 * i + c];
        });
      }
      grid.sync();
      if (fin) {
        products64(x);
        double v = 0.0;
        for_nodes([&](int i, int o) {
          for (int c = 0; c < 3; ++c) {
            const double t = a.b[3 * i + c] - acc[o + c];
            t64[3 * i + c] = t;
            v += t * t;
          }
        });
        write_norm(v);
      }
      grid.sync();
      scene_totals<1, double>(a, partD + myrep * (size_t)nblk, nblk, sh, nullptr);
      if (act == ACT_END) {  // decision threads of those scenes
        tt = scene_total(a, sh, 0, dsc);
        bool again = false;
        if (!isfinite(tt)) { status = 2; done = true; }
        else if (tt <= tol2_true || it >= a.max_iter || refine >= MAX_REFINE || !(tt > 0.0)) done = true;
        else {
          ++refine;
          begin_inner();
          again = true;
        }
        if (dsc == my_sc) sh.action = again ? 1 : 0;
      }
      __syncthreads();
      my_again = fin && sh.action;
      __syncthreads();
      init_inner(my_again);
    }
    grid.sync();
    my_run = my_act == ACT_STEP || my_again;
  }
  if (decider && status == 0 && !(tt <= tol2_true)) status = 3;
  report_solve(a, sh, decider, dsc, it, status, refine, decider && bb > 0.0 ? sqrt(fmax(tt, 0.0) / bb) : 0.0);
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

template <typename M>
static void* pcg_kernel(int rowg) {
  switch (rowg) {
    case 1: return (void*)k_pcg<M, 1>;
    case 2: return (void*)k_pcg<M, 2>;
    case 8: return (void*)k_pcg<M, 8>;
    default: return (void*)k_pcg<M, 4>;
  }
}

static void* pcg32_kernel(int rowg) {
  switch (rowg) {
    case 1: return (void*)k_pcg32<1>;
    case 2: return (void*)k_pcg32<2>;
    case 8: return (void*)k_pcg32<8>;
    default: return (void*)k_pcg32<4>;
  }
}

// fp32: the mixed-precision refinement solver; otherwise the FP64 pipelined solver
static void* pcg_fn(int fp32, int rowg) { return fp32 ? pcg32_kernel(rowg) : pcg_kernel<double>(rowg); }

int device_sms() {
  static std::mutex m;
  static std::vector<std::pair<int, int>> known;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(m);
  for (const auto& k : known)
    if (k.first == dev) return k.second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 1;
  known.push_back({dev, sms});
  return sms;
}

size_t pcg_smem_limit() {
  int dev, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return (size_t)optin;
}

// The dynamic shared-memory limit of a kernel is one process-wide setting per
// device.  Every PCG variant has it raised to the most the device allows next
// to the kernel's static shared memory, once, at its first use, and never
// lowered, so that simulators planning and launching on several host threads
// cannot change it under each other's launches.  Returns that limit (0 on
// failure).
static size_t ensure_smem_attr(void* f) {
  static std::mutex m;
  struct Entry { int dev; void* f; size_t limit; };
  static std::vector<Entry> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(m);
  for (const auto& d : done)
    if (d.dev == dev && d.f == f) return d.limit;
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) return 0;
  const size_t optin = pcg_smem_limit();
  const size_t limit = optin > fa.sharedSizeBytes ? optin - fa.sharedSizeBytes : 0;
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) != cudaSuccess) return 0;
  done.push_back({dev, f, limit});
  return limit;
}

int pcg_max_blocks(int threads, int fp32, int rowg, size_t dyn_smem) {
  int per_sm = 0;
  const int sms = device_sms();
  void* f = pcg_fn(fp32, rowg);
  if (dyn_smem > ensure_smem_attr(f)) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, dyn_smem) != cudaSuccess) return 0;
  return sms * per_sm;
}

cudaError_t launch_pcg(cudaStream_t st, int grid, int threads, const PcgArgs& a, int rowg, size_t dyn_smem) {
  void* args[] = {(void*)&a};
  count_launch();
  void* f = pcg_fn(a.fp32, rowg);
  if (dyn_smem > ensure_smem_attr(f)) return cudaErrorInvalidValue;
  return cudaLaunchCooperativeKernel(f, dim3(grid), dim3(threads), args, dyn_smem, st);
}

void launch_to_float(cudaStream_t st, size_t n, const double* src, float* dst, const int* n_dev, int stride) {
  if (!n) return;
  int grid = stride_grid((long long)n, 256, 16);
  k_to_float<<<grid, 256, 0, st>>>(n, src, dst, n_dev, stride);
  count_launch();
}

// Partition of the rows among the CTAs of a PCG launch (see PcgPlan).
namespace {
// n_parts contiguous cuts of [lo, hi) balanced by the prefix cost pre (pre[i] = cost of [0, i)); appends the
// n_parts - 1 inner boundaries and hi
void cut_balanced(const std::vector<long long>& pre, int lo, int hi, int n_parts, std::vector<int>& out) {
  int cur = lo;
  const long long c0 = pre[lo], tot = pre[hi] - c0;
  for (int c = 1; c < n_parts; ++c) {
    const long long target = c0 + tot * c / n_parts;
    while (cur < hi && pre[cur] < target) ++cur;
    out.push_back(cur);
  }
  out.push_back(hi);
}
// at least one part for every item of nonzero cost, the rest in proportion to the cost (largest remainders)
std::vector<int> share_parts(const std::vector<long long>& cost, int n_parts) {
  const int n = (int)cost.size();
  std::vector<int> k(n, 0);
  long long tot = 0;
  int used = 0;
  for (int s = 0; s < n; ++s)
    if (cost[s] > 0) { k[s] = 1; ++used; tot += cost[s]; }
  const int rest = n_parts - used;
  if (rest <= 0 || tot == 0) return k;
  std::vector<std::pair<long long, int>> frac;
  int given = 0;
  for (int s = 0; s < n; ++s) {
    if (!cost[s]) continue;
    const long long q = (long long)rest * cost[s];
    k[s] += (int)(q / tot);
    given += (int)(q / tot);
    frac.push_back({q % tot, s});
  }
  std::sort(frac.begin(), frac.end(), [](const std::pair<long long, int>& x, const std::pair<long long, int>& y) {
    return x.first != y.first ? x.first > y.first : x.second < y.second;
  });
  for (int j = 0; given < rest && j < (int)frac.size(); ++j, ++given) ++k[frac[j].second];
  return k;
}
}  // namespace

void pcg_plan_rows(const std::vector<int>& row, int nf, int nab, int grid, const std::vector<int>& node_scene,
                   int n_scenes, PcgPlan& P, const std::vector<int>* row_extra) {
  P.grid = grid;
  // FEM rows balanced by stored blocks plus a per-row cost (plus row_extra, the contact work of the row);
  // ABD bodies by count
  std::vector<long long> pre(nf + 1, 0);
  for (int i = 0; i < nf; ++i)
    pre[i + 1] = pre[i] + (row[i + 1] - row[i]) + 2 + (row_extra ? (long long)(*row_extra)[i] : 0);
  std::vector<long long> bpre(nab + 1);
  for (int b = 0; b <= nab; ++b) bpre[b] = b;

  // per-scene solves need the rows of every scene contiguous, a CTA of their own for each scene's FEM rows
  // and ABD bodies, and at most PCG_SCENES_MAX scenes
  std::vector<int> fem_lo, abd_lo;  // first row / body of every scene, then the end
  bool per_scene = n_scenes > 1 && n_scenes <= PCG_SCENES_MAX && (int)node_scene.size() >= nf + 4 * nab;
  if (per_scene) {
    fem_lo.assign(n_scenes + 1, nf);
    abd_lo.assign(n_scenes + 1, nab);
    int last = 0;
    for (int i = 0; i < nf && per_scene; ++i) {
      const int s = node_scene[i];
      if (s < last || s >= n_scenes) per_scene = false;
      else for (; last < s; ++last) fem_lo[last + 1] = i;
    }
    for (int s = 0; s <= n_scenes; ++s) if (s > last) fem_lo[s] = nf;
    fem_lo[0] = 0;
    last = 0;
    for (int b = 0; b < nab && per_scene; ++b) {
      const int s = node_scene[nf + 4 * b];
      if (s < last || s >= n_scenes) per_scene = false;
      else for (; last < s; ++last) abd_lo[last + 1] = b;
    }
    for (int s = 0; s <= n_scenes; ++s) if (s > last) abd_lo[s] = nab;
    abd_lo[0] = 0;
  }
  std::vector<long long> fcost, acost;
  int fem_scenes = 0, abd_scenes = 0;
  if (per_scene) {
    fcost.resize(n_scenes);
    acost.resize(n_scenes);
    for (int s = 0; s < n_scenes; ++s) {
      fcost[s] = pre[fem_lo[s + 1]] - pre[fem_lo[s]];
      acost[s] = abd_lo[s + 1] - abd_lo[s];
      fem_scenes += fcost[s] > 0;
      abd_scenes += acost[s] > 0;
    }
    P.n_abd_ctas = nab > 0 ? std::min(nab, std::max(abd_scenes, grid / 8)) : 0;
    P.n_fem_ctas = grid - P.n_abd_ctas;
    if (P.n_fem_ctas < std::max(1, fem_scenes)) per_scene = false;
  }
  if (!per_scene) {
    P.n_abd_ctas = nab > 0 ? std::min(nab, std::max(1, grid / 8)) : 0;
    P.n_fem_ctas = std::max(1, grid - P.n_abd_ctas);
    if (P.n_fem_ctas + P.n_abd_ctas > grid) P.n_abd_ctas = grid - P.n_fem_ctas;
  }
  P.seg.assign(1, 0);
  P.abd_seg.assign(1, 0);
  P.cta_scene.assign(grid, -1);
  if (per_scene) {
    P.n_psc = n_scenes;
    const std::vector<int> kf = share_parts(fcost, P.n_fem_ctas), ka = share_parts(acost, P.n_abd_ctas);
    int c = 0;
    for (int s = 0; s < n_scenes; ++s) {
      if (!kf[s]) continue;
      cut_balanced(pre, fem_lo[s], fem_lo[s + 1], kf[s], P.seg);
      for (int j = 0; j < kf[s]; ++j) P.cta_scene[c++] = s;
    }
    while (c < P.n_fem_ctas) { P.seg.push_back(nf); ++c; }  // spare CTAs: no rows, no scene
    c = 0;
    for (int s = 0; s < n_scenes; ++s) {
      if (!ka[s]) continue;
      cut_balanced(bpre, abd_lo[s], abd_lo[s + 1], ka[s], P.abd_seg);
      for (int j = 0; j < ka[s]; ++j) P.cta_scene[P.n_fem_ctas + c++] = s;
    }
    while (c < P.n_abd_ctas) { P.abd_seg.push_back(nab); ++c; }
  } else {
    P.n_psc = 1;
    cut_balanced(pre, 0, nf, P.n_fem_ctas, P.seg);
    if (P.n_abd_ctas) cut_balanced(bpre, 0, nab, P.n_abd_ctas, P.abd_seg);
    for (int c = 0; c < grid; ++c) P.cta_scene[c] = 0;  // every CTA takes part in the one solve
  }
  // CTAs of every scene, in CTA order
  P.sc_ptr.assign(P.n_psc + 1, 0);
  for (int c = 0; c < grid; ++c)
    if (P.cta_scene[c] >= 0) ++P.sc_ptr[P.cta_scene[c] + 1];
  for (int s = 0; s < P.n_psc; ++s) P.sc_ptr[s + 1] += P.sc_ptr[s];
  P.sc_cta.assign(P.sc_ptr[P.n_psc], 0);
  {
    std::vector<int> fill(P.sc_ptr.begin(), P.sc_ptr.end() - 1);
    for (int c = 0; c < grid; ++c)
      if (P.cta_scene[c] >= 0) P.sc_cta[fill[P.cta_scene[c]]++] = c;
  }
  for (int b = 1; b <= nab; ++b) P.seg.push_back(nf + 4 * b);
  P.max_rows = 0;
  P.max_blocks = 0;
  for (int c = 0; c < P.n_fem_ctas; ++c) {
    P.max_rows = std::max(P.max_rows, P.seg[c + 1] - P.seg[c]);
    P.max_blocks = std::max(P.max_blocks, row[P.seg[c + 1]] - row[P.seg[c]]);
  }
  int bodies_per_cta = 0;
  for (int c = 0; c < P.n_abd_ctas; ++c) bodies_per_cta = std::max(bodies_per_cta, P.abd_seg[c + 1] - P.abd_seg[c]);
  P.acc_doubles = std::max(1, std::max(3 * P.max_rows, 12 * bodies_per_cta));
  P.acc_doubles = (P.acc_doubles + 1) & ~1;  // keeps what follows 16-byte aligned
}

size_t pcg_contact_bytes(const PcgPlan& P) { return (8 * (size_t)P.acc_doubles + 127) & ~(size_t)127; }

size_t pcg_resident_bytes(const PcgPlan& P, int fp32) {
  size_t e = fp32 ? 4 : 8;
  size_t b = 8 * (size_t)P.acc_doubles + 9 * (size_t)P.max_blocks * e + 9 * (size_t)P.max_rows * e +
             4 * (size_t)P.max_blocks + 4 * ((size_t)P.max_rows + 1);
  return (b + 127) & ~(size_t)127;
}

}  // namespace ipc
