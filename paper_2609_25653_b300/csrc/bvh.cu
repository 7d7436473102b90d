// LBVH construction and refit (see bvh.cuh).
#include <algorithm>
#include "bvh.cuh"
#include "kernels.h"

namespace ipc {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int BOUND_BLOCKS = 512;  // fan-in of the scene-bound reduction

// ---------------------------------------------------------------------------
// leaf boxes
// ---------------------------------------------------------------------------
__device__ inline void grow(double* b, d3 x) {
  b[0] = fmin(b[0], x.x); b[1] = fmin(b[1], x.y); b[2] = fmin(b[2], x.z);
  b[3] = fmax(b[3], x.x); b[4] = fmax(b[4], x.y); b[5] = fmax(b[5], x.z);
}

// Box of each triangle (nvp = 3) or edge (nvp = 2) over its vertices at x
// (and x + p when p != null), widened by pad on every side.
__global__ void k_leaf_boxes(int n, const int* __restrict__ ids, int nvp, const double* __restrict__ xv,
                             const double* __restrict__ pv, double pad, double* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  double b[6] = {inf, inf, inf, -inf, -inf, -inf};
  for (int q = 0; q < nvp; ++q) {
    int v = ids[nvp * k + q];
    d3 x = ld3(xv, v);
    grow(b, x);
    if (pv) grow(b, x + ld3(pv, v));
  }
  double* o = out + 6 * (size_t)k;
  o[0] = b[0] - pad; o[1] = b[1] - pad; o[2] = b[2] - pad;
  o[3] = b[3] + pad; o[4] = b[4] + pad; o[5] = b[5] + pad;
}

// scene bounds of the box centres: per-block partials, then one block
__global__ void k_bounds_partial(int n, const double* __restrict__ leaf, double* __restrict__ part) {
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  double lo[3] = {inf, inf, inf}, hi[3] = {-inf, -inf, -inf};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double* b = leaf + 6 * (size_t)k;
    for (int d = 0; d < 3; ++d) {
      double c = 0.5 * (b[d] + b[3 + d]);
      lo[d] = fmin(lo[d], c);
      hi[d] = fmax(hi[d], c);
    }
  }
  for (int d = 0; d < 3; ++d) {
    double m = block_max(-lo[d]);
    if (threadIdx.x == 0) part[6 * blockIdx.x + d] = -m;
    m = block_max(hi[d]);
    if (threadIdx.x == 0) part[6 * blockIdx.x + 3 + d] = m;
  }
}

__global__ void k_bounds_final(int nblk, double* __restrict__ part) {
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  double lo[3] = {inf, inf, inf}, hi[3] = {-inf, -inf, -inf};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(lo[d], part[6 * b + d]);
      hi[d] = fmax(hi[d], part[6 * b + 3 + d]);
    }
  for (int d = 0; d < 3; ++d) {
    double m = block_max(-lo[d]);
    double h = block_max(hi[d]);
    if (threadIdx.x == 0) {
      part[6 * nblk + d] = -m;
      part[6 * nblk + 3 + d] = h;
    }
  }
}

__device__ inline unsigned spread10(unsigned v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void k_morton(int n, const double* __restrict__ leaf, const double* __restrict__ bounds,
                         unsigned* __restrict__ codes, int* __restrict__ prim) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double* b = leaf + 6 * (size_t)k;
  unsigned q[3];
  for (int d = 0; d < 3; ++d) {
    double ext = bounds[3 + d] - bounds[d];
    double u = ext > 0.0 ? (0.5 * (b[d] + b[3 + d]) - bounds[d]) / ext : 0.0;
    u = fmin(fmax(u, 0.0), 1.0);
    q[d] = min(1023u, (unsigned)(u * 1024.0));
  }
  codes[k] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
  prim[k] = k;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (code, prim) by code, 8-bit digits
// ---------------------------------------------------------------------------
__global__ void k_radix_hist(int n, const unsigned* __restrict__ keys, int shift, int nblk, int* __restrict__ hist) {
  __shared__ int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  int base = blockIdx.x * SORT_TILE;
  for (int i = threadIdx.x; i < SORT_TILE; i += blockDim.x) {
    int e = base + i;
    if (e < n) atomicAdd(&h[(keys[e] >> shift) & 255u], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d * nblk + blockIdx.x] = h[d];
}

// exclusive scan of m ints in place, one block of 1024 threads
__global__ void k_scan(int m, int* __restrict__ a) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < m; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < m ? a[i] : 0;
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
    int incl = x + (w > 0 ? warp_tot[w - 1] : 0) + carry;
    if (i < m) a[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
}

__global__ void k_radix_scatter(int n, const unsigned* __restrict__ keys, const int* __restrict__ vals, int shift,
                                int nblk, const int* __restrict__ offs, unsigned* __restrict__ keys_out,
                                int* __restrict__ vals_out) {
  __shared__ int base[256];
  __shared__ int wcnt[SORT_THREADS / 32][256];
  __shared__ int ctot[256];
  const int nw = SORT_THREADS / 32;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < 256; d += blockDim.x) base[d] = offs[d * nblk + blockIdx.x];
  int tile0 = blockIdx.x * SORT_TILE;
  for (int chunk = 0; chunk < SORT_ITEMS; ++chunk) {
    for (int i = threadIdx.x; i < nw * 256; i += blockDim.x) wcnt[i / 256][i % 256] = 0;
    __syncthreads();
    int e = tile0 + chunk * SORT_THREADS + threadIdx.x;
    bool valid = e < n;
    unsigned key = valid ? keys[e] : 0u;
    int d = valid ? (int)((key >> shift) & 255u) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) {
      int run = 0;
      for (int q = 0; q < nw; ++q) {
        int t = wcnt[q][dd];
        wcnt[q][dd] = run;
        run += t;
      }
      ctot[dd] = run;
    }
    __syncthreads();
    if (valid) {
      int pos = base[d] + wcnt[w][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = vals[e];
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) base[dd] += ctot[dd];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// hierarchy (Karras 2012)
// ---------------------------------------------------------------------------
__device__ inline int delta(const unsigned* codes, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  unsigned a = codes[i], b = codes[j];
  if (a != b) return __clz(a ^ b);
  return 32 + __clz((unsigned)(i ^ j));
}

__global__ void k_hierarchy(int n, const unsigned* __restrict__ codes, int* __restrict__ left, int* __restrict__ right,
                            int* __restrict__ parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int dir = (delta(codes, n, i, i + 1) - delta(codes, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(codes, n, i, i - dir);
  int lmax = 2;
  while (delta(codes, n, i, i + lmax * dir) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(codes, n, i, i + (l + t) * dir) > dmin) l += t;
  int j = i + l * dir;
  int dnode = delta(codes, n, i, j);
  int s = 0;
  for (int div = 2;; div <<= 1) {
    int t = (l + div - 1) / div;
    if (delta(codes, n, i, i + (s + t) * dir) > dnode) s += t;
    if (t <= 1) break;
  }
  int gamma = i + s * dir + min(dir, 0);
  int lo = min(i, j), hi = max(i, j);
  int lc = (lo == gamma) ? (n - 1 + gamma) : gamma;
  int rc = (hi == gamma + 1) ? (n - 1 + gamma + 1) : gamma + 1;
  left[i] = lc;
  right[i] = rc;
  parent[lc] = i;
  parent[rc] = i;
  if (i == 0) parent[0] = -1;
}

// leaf boxes to nodes, then up the tree: the second child to arrive merges
__global__ void k_refit(int n, const int* __restrict__ prim, const double* __restrict__ leaf,
                        const int* __restrict__ left, const int* __restrict__ right, const int* __restrict__ parent,
                        int* __restrict__ flag, float* __restrict__ box) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int node = n - 1 + k;
  box_outward(leaf + 6 * (size_t)prim[k], box + 6 * (size_t)node);
  if (n == 1) return;
  int p = parent[node];
  while (p >= 0) {
    __threadfence();
    if (atomicAdd(flag + p, 1) == 0) return;
    __threadfence();
    const volatile float* a = box + 6 * (size_t)left[p];
    const volatile float* b = box + 6 * (size_t)right[p];
    float* o = box + 6 * (size_t)p;
    o[0] = fminf(a[0], b[0]); o[1] = fminf(a[1], b[1]); o[2] = fminf(a[2], b[2]);
    o[3] = fmaxf(a[3], b[3]); o[4] = fmaxf(a[4], b[4]); o[5] = fmaxf(a[5], b[5]);
    p = parent[p];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int nb(int n, int t) { return (n + t - 1) / t; }

// Sizes of the arrays of a tree of capacity c (the order of Bvh's pointers).
static void bvh_sizes(int c, size_t out[12]) {
  const int nblk = nb(c, SORT_TILE);
  const size_t sz[12] = {sizeof(unsigned) * c, sizeof(int) * c, sizeof(unsigned) * c, sizeof(int) * c,
                         sizeof(int) * c, sizeof(int) * c, sizeof(int) * 2 * (size_t)c, sizeof(int) * c,
                         sizeof(float) * 6 * 2 * (size_t)c, sizeof(double) * 6 * (size_t)c, sizeof(int) * 256 * (size_t)nblk,
                         sizeof(double) * 6 * (BOUND_BLOCKS + 1)};
  for (int i = 0; i < 12; ++i) out[i] = sz[i];
}

static void** bvh_ptr(Bvh& B, int i) {
  void** p[12] = {(void**)&B.codes, (void**)&B.prim, (void**)&B.codes_tmp, (void**)&B.prim_tmp, (void**)&B.left,
                  (void**)&B.right, (void**)&B.parent, (void**)&B.flag, (void**)&B.box, (void**)&B.leafbox,
                  (void**)&B.hist, (void**)&B.bounds};
  return p[i];
}

void bvh_free(Bvh& B, DevAlloc& mem) {
  size_t sz[12];
  bvh_sizes(B.cap, sz);
  for (int i = 0; i < 12; ++i) mem.put(*bvh_ptr(B, i), sz[i]);
  B = Bvh{};
}

cudaError_t bvh_alloc(Bvh& B, int n, DevAlloc& mem) {
  if (n <= B.cap && B.codes) { B.n = n; return cudaSuccess; }
  bvh_free(B, mem);
  B.n = n;
  const int c = std::max(n, 1);
  size_t sz[12];
  bvh_sizes(c, sz);
  B.cap = c;
  B.hist_cap = 256 * nb(c, SORT_TILE);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 12 && e == cudaSuccess; ++i) e = mem.get(bvh_ptr(B, i), sz[i]);
  return e;
}

void bvh_leaf_boxes(cudaStream_t st, Bvh& B, const int* ids, int nvp, const double* xv, const double* pv, double pad) {
  if (B.n <= 0) return;
  k_leaf_boxes<<<nb(B.n, 256), 256, 0, st>>>(B.n, ids, nvp, xv, pv, pad, B.leafbox);
  count_launch();
}

void bvh_refit(cudaStream_t st, Bvh& B) {
  if (B.n <= 0) return;
  if (B.n > 1) cudaMemsetAsync(B.flag, 0, sizeof(int) * (B.n - 1), st);
  k_refit<<<nb(B.n, 256), 256, 0, st>>>(B.n, B.prim, B.leafbox, B.left, B.right, B.parent, B.flag, B.box);
  count_launch();
}

// Sort the leaves by Morton code of the current leaf boxes and rebuild the hierarchy, then refit.
void bvh_build(cudaStream_t st, Bvh& B) {
  int n = B.n;
  if (n <= 0) return;
  int pb = std::min(BOUND_BLOCKS, nb(n, 256));
  k_bounds_partial<<<pb, 256, 0, st>>>(n, B.leafbox, B.bounds);
  k_bounds_final<<<1, 256, 0, st>>>(pb, B.bounds);
  k_morton<<<nb(n, 256), 256, 0, st>>>(n, B.leafbox, B.bounds + 6 * pb, B.codes, B.prim);
  count_launch(3);
  int nblk = nb(n, SORT_TILE);
  unsigned *ka = B.codes, *kb = B.codes_tmp;
  int *va = B.prim, *vb = B.prim_tmp;
  for (int shift = 0; shift < 32; shift += 8) {
    k_radix_hist<<<nblk, SORT_THREADS, 0, st>>>(n, ka, shift, nblk, B.hist);
    k_scan<<<1, 1024, 0, st>>>(256 * nblk, B.hist);
    k_radix_scatter<<<nblk, SORT_THREADS, 0, st>>>(n, ka, va, shift, nblk, B.hist, kb, vb);
    count_launch(3);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  // four passes: sorted data is back in codes / prim
  if (n > 1) {
    k_hierarchy<<<nb(n - 1, 256), 256, 0, st>>>(n, B.codes, B.left, B.right, B.parent);
    count_launch();
  } else {
    cudaMemsetAsync(B.parent, 0xff, sizeof(int), st);
  }
  bvh_refit(st, B);
}

}  // namespace ipc
