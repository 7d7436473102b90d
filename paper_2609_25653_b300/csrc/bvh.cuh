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
  double* box = nullptr;     // (2 cap, 6) lo.xyz, hi.xyz
  double* leafbox = nullptr; // (cap, 6) primitive boxes in primitive order
  int* hist = nullptr;       // radix histograms
  int hist_cap = 0;
  double* bounds = nullptr;  // (2 * 148 * 8, 6) partial scene bounds
};

__device__ inline bool box_overlap(const double* a, const double* b) {
  return !(a[0] > b[3] || b[0] > a[3] || a[1] > b[4] || b[1] > a[4] || a[2] > b[5] || b[2] > a[5]);
}

}  // namespace ipc
