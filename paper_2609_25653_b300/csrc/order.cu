// Canonical order of the lists built with atomic appends.
//
// Culling appends contact pairs, and the ABD coupling pass appends its
// per-pair blocks, in whatever order the threads reach their atomic
// counters.  Every later sum over such a list (the contact rows of the PCG,
// the friction data, the per-body coupling rows) would then be formed in a
// different order in every run.  The lists are therefore put into a canonical
// order right after they are built: a stable least-significant-digit radix
// sort (8-bit digits) of 64-bit keys with an index payload, whose length is
// read on the device (the host does not know it before the next
// synchronisation), then a gather of the records by the sorted index.
#include <utility>
#include "common.cuh"
#include "kernels.h"

namespace ipc {

namespace {

constexpr int OT = 256;                 // threads per sorting block
constexpr int OITEMS = 8;               // items per thread and tile
constexpr int OTILE = OT * OITEMS;

__device__ inline int list_len(const int* n_dev, int cap) { return min(*n_dev, cap); }

// digit histogram of every tile: hist[d * nblk + tile]
__global__ void __launch_bounds__(OT) k_hist(const int* __restrict__ n_dev, int cap,
                                             const unsigned long long* __restrict__ keys, int shift, int nblk,
                                             int* __restrict__ hist) {
  __shared__ int h[256];
  const int n = list_len(n_dev, cap);
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int base = blockIdx.x * OTILE;
  for (int i = threadIdx.x; i < OTILE; i += blockDim.x) {
    const int e = base + i;
    if (e < n) atomicAdd(&h[(int)((keys[e] >> shift) & 255ull)], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d * nblk + blockIdx.x] = h[d];
}

// stable scatter of every tile to the scanned digit offsets: items of equal digit keep their order
// (thread order within a chunk of OT items, chunks in order)
__global__ void __launch_bounds__(OT) k_scatter(const int* __restrict__ n_dev, int cap,
                                                const unsigned long long* __restrict__ keys,
                                                const int* __restrict__ vals, int shift, int nblk,
                                                const int* __restrict__ offs, unsigned long long* __restrict__ keys_out,
                                                int* __restrict__ vals_out) {
  __shared__ int base[256];
  __shared__ int wcnt[OT / 32][256];
  __shared__ int ctot[256];
  const int n = list_len(n_dev, cap);
  const int tile0 = blockIdx.x * OTILE;
  if (tile0 >= n) return;  // whole block leaves together
  const int nw = OT / 32, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < 256; d += blockDim.x) base[d] = offs[d * nblk + blockIdx.x];
  for (int chunk = 0; chunk < OITEMS; ++chunk) {
    for (int i = threadIdx.x; i < nw * 256; i += blockDim.x) wcnt[i / 256][i % 256] = 0;
    __syncthreads();
    const int e = tile0 + chunk * OT + threadIdx.x;
    const bool valid = e < n;
    const unsigned long long key = valid ? keys[e] : 0ull;
    const int d = valid ? (int)((key >> shift) & 255ull) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) {
      int run = 0;
      for (int q = 0; q < nw; ++q) {
        const int t = wcnt[q][dd];
        wcnt[q][dd] = run;
        run += t;
      }
      ctot[dd] = run;
    }
    __syncthreads();
    if (valid) {
      const int pos = base[d] + wcnt[w][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = vals[e];
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) base[dd] += ctot[dd];
    __syncthreads();
  }
}

// key of a contact pair: (kind, primitive a, primitive b), unique within one list
__global__ void k_pair_keys(const int* __restrict__ n_dev, int cap, const int* __restrict__ rec, int bits,
                            unsigned long long* __restrict__ keys, int* __restrict__ idx) {
  const int n = list_len(n_dev, cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int* r = rec + 8 * (size_t)i;
    keys[i] = ((unsigned long long)r[0] << (2 * bits)) | ((unsigned long long)(unsigned)r[1] << bits) |
              (unsigned long long)(unsigned)r[2];
    idx[i] = i;
  }
}

__global__ void k_gather_pairs(const int* __restrict__ n_dev, int cap, const int* __restrict__ idx,
                               const int* __restrict__ rec_in, const double* __restrict__ s_in, int* __restrict__ rec,
                               double* __restrict__ s) {
  const int n = list_len(n_dev, cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int j = idx[i];
    const int* src = rec_in + 8 * (size_t)j;
    int* dst = rec + 8 * (size_t)i;
    for (int c = 0; c < 8; ++c) dst[c] = src[c];
    if (s) s[i] = s_in[j];
  }
}

}  // namespace

size_t sort_hist_ints(int cap) { return 256 * (size_t)((cap + OTILE - 1) / OTILE) + 1; }

void launch_sort_u64(cudaStream_t st, const int* n_dev, int cap, int key_bits, unsigned long long* keys, int* idx,
                     unsigned long long* keys_tmp, int* idx_tmp, int* hist, int* scan_tiles) {
  if (cap <= 0) return;
  const int nblk = (cap + OTILE - 1) / OTILE;
  const int passes = (key_bits + 7) / 8;
  unsigned long long *ka = keys, *kb = keys_tmp;
  int *va = idx, *vb = idx_tmp;
  for (int p = 0; p < passes; ++p) {
    k_hist<<<nblk, OT, 0, st>>>(n_dev, cap, ka, 8 * p, nblk, hist);
    launch_scan_exclusive(st, 256 * nblk, hist, scan_tiles);
    k_scatter<<<nblk, OT, 0, st>>>(n_dev, cap, ka, va, 8 * p, nblk, hist, kb, vb);
    count_launch(2);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (passes & 1) {
    // the result sits in the scratch buffers: copy it back (lengths up to cap; only the first n are used)
    cudaMemcpyAsync(keys, ka, sizeof(unsigned long long) * (size_t)cap, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(idx, va, sizeof(int) * (size_t)cap, cudaMemcpyDeviceToDevice, st);
  }
}

void launch_sort_pairs(cudaStream_t st, const int* n_dev, int cap, int prim_bits, int* rec, double* rec_s,
                       const OrderWork& W) {
  if (cap <= 0) return;
  const int grid = stride_grid(cap, 256, 8);
  k_pair_keys<<<grid, 256, 0, st>>>(n_dev, cap, rec, prim_bits, W.keys, W.idx);
  count_launch();
  launch_sort_u64(st, n_dev, cap, 2 * prim_bits + 1, W.keys, W.idx, W.keys_tmp, W.idx_tmp, W.hist, W.tiles);
  cudaMemcpyAsync(W.rec_tmp, rec, sizeof(int) * 8 * (size_t)cap, cudaMemcpyDeviceToDevice, st);
  if (rec_s) cudaMemcpyAsync(W.s_tmp, rec_s, sizeof(double) * (size_t)cap, cudaMemcpyDeviceToDevice, st);
  k_gather_pairs<<<grid, 256, 0, st>>>(n_dev, cap, W.idx, W.rec_tmp, rec_s ? W.s_tmp : nullptr, rec, rec_s);
  count_launch();
}

}  // namespace ipc
