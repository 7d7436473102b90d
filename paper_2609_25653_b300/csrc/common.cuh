// Shared device-side declarations of the ipcsim CUDA library (sm_103a).
//
// Layouts (all double unless stated):
//   vertices  : global order [FEM | ABD surface | kinematic], positions AoS (nv, 3)
//   nodes     : 3-DOF groups [FEM vertex i -> node i | ABD body b -> nodes nf+4b .. nf+4b+3]
//               (ABD pseudo-nodes: translation p, then the columns of A)
//   DOF vector: (n_nodes, 3), free DOFs only; kinematic vertices are Dirichlet
//   BSR 3x3   : row_ptr (n_nodes+1), col (nnzb), val (nnzb, 9) row-major blocks,
//               full (both triangles stored)
//   pairs     : int rec[8] = kind (0 PT / 1 EE), prim a, prim b, type, v0..v3
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace ipc {

constexpr int VK_FEM = 0, VK_ABD = 1, VK_KIN = 2;

// Read-only scene topology and material data on the device.
struct DevScene {
  int nf, nt, nab, nkb, nv, na_v, nk, n_nodes;
  int nsv, ntri, nedge, nbody;
  const int4* tets;          // (nt)
  const double* B;           // (nt, 9) Dm^-1 row-major
  const double* vol;         // (nt)
  const double* mu;          // (nt)
  const double* lam;         // (nt) model parameter (first Lame + mu)
  const int* tet_blk;        // (nt, 16) BSR block of (a, b)
  const int* vkind;          // (nv)
  const int* vbody;          // (nv) body id (FEM bodies, then ABD, then kinematic)
  const int* vabd;           // (nv) ABD body index for ABD vertices, else -1
  const double* xbar;        // (nv, 3) body-frame rest position (ABD), local (kinematic), rest (FEM)
  const int* bkind;          // (nbody)
  const int* sv;             // (nsv) surface vertex ids
  const int3* tris;          // (ntri)
  const int2* edges;         // (nedge)
  const double* edge_rest_sq;// (nedge)
  const double* node_mass;   // (nf) FEM lumped masses
  const double* abd_S;       // (nab, 16) rho * int phi phi^T, phi = (1, xbar)
  const double* abd_vol;     // (nab)
  const int* abd_blk;        // (nab, 16) BSR blocks of the 4x4 pseudo-node grid
  const int* kin_vbody;      // (nk) kinematic body of each kinematic vertex (0-based among kinematic)
  int n_stitch;
  const int* stitch_v;
  const int* stitch_b;
  const double* stitch_X;    // (n_stitch, 3)
  // joint drives between affine bodies: side a (sign +) and b (sign -), body -1 = the world
  int nj;
  const int* jt_body;        // (nj, 2)
  const int* jt_kind;        // (nj, 2) 0 body-frame point, 1 body-frame direction
  const double* jt_va;       // (nj, 3) vector on side a
  const double* jt_vb;       // (nj, 3) vector on side b (set per step)
  const double* jt_k;        // (nj)
  const double* jt_t;        // (nj, 3) target offset (set per step)
  const int* jt_blk;         // (nj, 64) BSR block of pseudo-node pair (4 s + m, 4 s' + n), -1 for the world
  const int* bsr_row;        // (n_nodes + 1)
  const int* bsr_col;        // (nnzb)
  const int* bsr_diag;       // (n_nodes) index of the diagonal block
  int nnzb;
  // independent scenes of a batch: scene of every body, per-scene barrier and stitch stiffness
  int n_scenes;
  const int* body_scene;     // (nbody)
  const double* scene_kappa; // (n_scenes)
  const double* scene_kc;    // (n_scenes)
  // per-scene Newton control of a batch (null for a single scene): scene of every
  // node, energy terms per scene (n_scenes, 8), CCD bound per scene (double bits),
  // max |p_F| and max |p_D| per scene (double bits), line-search step per scene
  const int* node_scene;
  double* E_sc;
  unsigned long long* alpha_sc;
  unsigned long long* pn_sc;
  const double* alpha_trial;
};

__device__ inline int scene_of_vertex(const DevScene& S, int v) { return S.body_scene[S.vbody[v]]; }

// energy term comp of one element of scene sc (batches only)
__device__ inline void scene_energy(const DevScene& S, int sc, int comp, double e) {
  if (S.E_sc && e != 0.0) atomicAdd(S.E_sc + 8 * sc + comp, e);
}

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
struct d3 { double x, y, z; };
__host__ __device__ inline d3 mk(double a, double b, double c) { return d3{a, b, c}; }
__host__ __device__ inline d3 operator+(d3 a, d3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__host__ __device__ inline d3 operator-(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ inline d3 operator*(double s, d3 a) { return {s * a.x, s * a.y, s * a.z}; }
__host__ __device__ inline double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline d3 cross(d3 a, d3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ inline d3 ld3(const double* p, int i) { return {p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
__device__ inline void st3(double* p, int i, d3 v) { p[3 * i] = v.x; p[3 * i + 1] = v.y; p[3 * i + 2] = v.z; }
__device__ inline double comp(d3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

// order-preserving encoding of non-negative doubles for atomicMin
__device__ inline unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

// block-wide sum (blockDim.x multiple of 32, <= 1024); result valid in thread 0
__device__ inline double block_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline double block_max(double v) {
  __shared__ double shm[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) shm[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? shm[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Map of a vertex to its DOF nodes: up to 4 (node, weight) entries.
struct NodeMap { int n; int node[4]; double w[4]; };
__device__ inline NodeMap vertex_nodes(const DevScene& S, int v) {
  NodeMap m;
  int k = S.vkind[v];
  if (k == VK_FEM) { m.n = 1; m.node[0] = v; m.w[0] = 1.0; }
  else if (k == VK_ABD) {
    int b = S.vabd[v];
    m.n = 4;
    int base = S.nf + 4 * b;
    m.node[0] = base; m.w[0] = 1.0;
    m.node[1] = base + 1; m.w[1] = S.xbar[3 * v];
    m.node[2] = base + 2; m.w[2] = S.xbar[3 * v + 1];
    m.node[3] = base + 3; m.w[3] = S.xbar[3 * v + 2];
  } else m.n = 0;
  return m;
}

// error flag bits written by kernels
enum : int { ERRF_BVH = 1, ERRF_PCG_BREAK = 2, ERRF_NAN = 4, ERRF_PAIR_OVF = 8, ERRF_FRIC_OVF = 16, ERRF_INC = 32,
             ERRF_ABD = 64 };

}  // namespace ipc
