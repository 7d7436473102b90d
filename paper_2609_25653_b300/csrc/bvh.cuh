// Linear BVH over primitive boxes: Morton codes of box centres, a stable LSD
// radix sort, the hierarchy of Karras ("Maximizing Parallelism in the
// Construction of BVHs, Octrees, and k-d Trees", HPG 2012) and an atomic
// bottom-up refit.  Internal nodes 0..n-2, leaf k is node n-1+k.
#pragma once
#include "common.cuh"

namespace ipc {

struct Bvh {
  int n = 0;                 // primitives
  int cap = 0;               // allocated primitives
  unsigned* codes = nullptr; // (cap) sorted Morton codes
  int* prim = nullptr;       // (cap) primitive of each leaf (sorted order)
  unsigned* codes_tmp = nullptr;
  int* prim_tmp = nullptr;
  int* left = nullptr;       // (cap) children of internal nodes (node ids)
  int* right = nullptr;
  int* parent = nullptr;     // (2 cap)
  int* flag = nullptr;       // (cap) refit arrival counters
  float* box = nullptr;      // (2 cap, 6) node boxes lo.xyz, hi.xyz, rounded outward to FP32
  double* leafbox = nullptr; // (cap, 6) primitive boxes in primitive order
  int* hist = nullptr;       // radix histograms
  int hist_cap = 0;
  double* bounds = nullptr;  // (partial blocks + 1, 6) partial scene bounds
};

__device__ inline bool box_overlap(const double* a, const double* b) {
  return !(a[0] > b[3] || b[0] > a[3] || a[1] > b[4] || b[1] > a[4] || a[2] > b[5] || b[2] > a[5]);
}

// The tree's node boxes are FP32 with lower bounds rounded down and upper bounds
// rounded up, so they contain the exact FP64 boxes: a traversal with an
// outward-rounded query visits every leaf the FP64 test would (and possibly a
// few more, which the exact tests after it reject).  FP32 compares issue at
// full rate on this part; FP64 ones do not.
__device__ inline bool box_overlap(const float* a, const float* b) {
  return !(a[0] > b[3] || b[0] > a[3] || a[1] > b[4] || b[1] > a[4] || a[2] > b[5] || b[2] > a[5]);
}
__device__ inline void box_outward(const double* d, float* f) {
  f[0] = __double2float_rd(d[0]); f[1] = __double2float_rd(d[1]); f[2] = __double2float_rd(d[2]);
  f[3] = __double2float_ru(d[3]); f[4] = __double2float_ru(d[4]); f[5] = __double2float_ru(d[5]);
}

}  // namespace ipc
