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

// error flag bits written by kernels
enum : int { ERRF_BVH = 1, ERRF_PCG_BREAK = 2, ERRF_NAN = 4, ERRF_PAIR_OVF = 8, ERRF_FRIC_OVF = 16, ERRF_INC = 32,
             ERRF_ABD = 64, ERRF_ACC = 128 };

// order-preserving encoding of non-negative doubles for atomicMin
__device__ inline unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

// ---------------------------------------------------------------------------
// Order-independent accumulation.  Every sum that many threads add into
// (energies, gradient, Hessian blocks, Dirichlet couplings, the coarse
// matrix) is kept as an exact 192-bit two's-complement fixed-point number
// with resolution 2^-ACC_FRAC (three 64-bit words, least significant first).
// A double is converted exactly (bits below 2^-ACC_FRAC are dropped, toward
// zero) and added with integer atomics whose carries are propagated word by
// word; integer addition is associative, so the words after a set of
// contributions do not depend on their order, and acc_value rounds the exact
// sum to the nearest double once.  Contributions of magnitude >= 2^ACC_MAX
// (or not finite) are not added and raise ERRF_ACC in *err.
// ---------------------------------------------------------------------------
using acc_t = unsigned long long;
constexpr int ACC_FRAC = 96;  // resolution 2^-96 ~ 1.3e-29
constexpr int ACC_MAX = 94;   // |x| < 2^94 ~ 2e28 per contribution
constexpr int E_SLOTS = 32;

// x as three words (w0 least significant) of x * 2^ACC_FRAC truncated toward zero; false if out of range
__host__ __device__ inline bool acc_words(double x, acc_t w[3]) {
  w[0] = w[1] = w[2] = 0;
  union { double d; acc_t u; } cv;
  cv.d = x;
  const int ex = (int)((cv.u >> 52) & 0x7ff);
  if (ex == 0) return true;        // zero or subnormal: below the resolution
  if (ex == 0x7ff) return false;   // inf / nan
  acc_t man = (cv.u & ((1ull << 52) - 1)) | (1ull << 52);  // |x| = man * 2^(ex - 1075)
  int sh = ex - 1075 + ACC_FRAC;
  if (ex - 1023 >= ACC_MAX) return false;
  if (sh < 0) {
    if (sh <= -53) return true;
    man >>= -sh;
    sh = 0;
  }
  // man < 2^53 placed at bit sh (sh <= ACC_FRAC + ACC_MAX - 53 < 192 - 53)
  const int q = sh >> 6, r = sh & 63;
  acc_t lo = man << r, hi = r ? (man >> (64 - r)) : 0;
  if (q == 0) { w[0] = lo; w[1] = hi; }
  else if (q == 1) { w[1] = lo; w[2] = hi; }
  else { w[2] = lo; }
  if (cv.u >> 63) {  // two's complement
    w[0] = ~w[0]; w[1] = ~w[1]; w[2] = ~w[2];
    if (++w[0] == 0 && ++w[1] == 0) ++w[2];
  }
  return true;
}

// three words (least significant first) added into a, carries propagated
__device__ inline void acc_add_words(acc_t* a, const acc_t w[3]) {
  acc_t c1 = 0;
  if (w[0]) {
    const acc_t o = atomicAdd(a, w[0]);
    c1 = (o + w[0] < o) ? 1ull : 0ull;
  }
  acc_t t1 = w[1] + c1, c2 = (t1 < w[1]) ? 1ull : 0ull;
  if (t1) {
    const acc_t o = atomicAdd(a + 1, t1);
    c2 += (o + t1 < o) ? 1ull : 0ull;
  }
  const acc_t t2 = w[2] + c2;
  if (t2) atomicAdd(a + 2, t2);
}

__device__ inline void acc_add(acc_t* a, double x, int* err = nullptr) {
  acc_t w[3];
  if (!acc_words(x, w)) {
    if (err) atomicOr(err, ERRF_ACC);
    return;
  }
  acc_add_words(a, w);
}

// exact sum of n accumulators (plain loads; the caller orders it after their writers)
__device__ inline void acc_sum_words(const acc_t* a, int n, acc_t w[3]) {
  w[0] = w[1] = w[2] = 0;
  for (int k = 0; k < n; ++k) {
    const acc_t s0 = a[3 * k], s1 = a[3 * k + 1], s2 = a[3 * k + 2];
    const acc_t t0 = w[0] + s0, c0 = t0 < w[0] ? 1ull : 0ull;
    const acc_t t1 = w[1] + s1, c1a = t1 < w[1] ? 1ull : 0ull;
    const acc_t t1c = t1 + c0, c1b = t1c < t1 ? 1ull : 0ull;
    w[0] = t0;
    w[1] = t1c;
    w[2] = w[2] + s2 + c1a + c1b;
  }
}

// the exact sum held in a rounded to the nearest double
__host__ __device__ inline double acc_value(const acc_t* a) {
  acc_t w0 = a[0], w1 = a[1], w2 = a[2];
  const bool neg = (w2 >> 63) != 0;
  if (neg) {
    w0 = ~w0; w1 = ~w1; w2 = ~w2;
    if (++w0 == 0 && ++w1 == 0) ++w2;
  }
  // the top 64 significant bits with a sticky bit for everything below, then one rounding to 53 bits
  acc_t top, rest;
  int e;  // value = top * 2^(e - ACC_FRAC)
  auto lead = [](acc_t v) {  // leading zero bits of v != 0
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return __builtin_clzll(v);
#endif
  };
  if (w2) {
    const int z = lead(w2);
    top = z ? (w2 << z) | (w1 >> (64 - z)) : w2;
    rest = z ? ((w1 << z) | w0) : (w1 | w0);
    e = 128 - z;
  } else if (w1) {
    const int z = lead(w1);
    top = z ? (w1 << z) | (w0 >> (64 - z)) : w1;
    rest = z ? (w0 << z) : w0;
    e = 64 - z;
  } else {
    top = w0;
    rest = 0;
    e = 0;
  }
  if (top == 0) return 0.0;
  if (rest) top |= 1ull;  // sticky: below the 11 bits dropped by the conversion
  double v = (double)top;  // round to nearest even
  // scale by 2^(e - ACC_FRAC) exactly (power of two, normal range)
  union { double d; acc_t u; } s;
  s.u = (acc_t)(1023 + e - ACC_FRAC) << 52;
  v *= s.d;
  return neg ? -v : v;
}

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
  // elastic gathers: the FEM BSR blocks (the first nfb) with their tets (code tet << 4 | a << 2 | b, in tet
  // order), and every FEM node with its tets (code tet << 2 | a)
  int nfb;
  const int* eg_blk_ptr;
  const int* eg_blk_ent;
  const int* eg_node_ptr;
  const int* eg_node_ent;
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
  acc_t* E_sc;               // (n_scenes, 8) accumulators
  int* err;                  // error flags of the iteration (ERRF_*)
  acc_t* e_slots;            // (E_SLOTS) accumulators spreading one energy sum over many addresses
  unsigned long long* min_sc;  // batches: smallest squared distance of every scene's assembly (double bits)
  unsigned long long* alpha_sc;
  unsigned long long* pn_sc;
  const double* alpha_trial;
};

__device__ inline int scene_of_vertex(const DevScene& S, int v) { return S.body_scene[S.vbody[v]]; }

// energy term comp of one element of scene sc (batches only)
__device__ inline void scene_energy(const DevScene& S, int sc, int comp, double e) {
  if (S.E_sc && e != 0.0) acc_add(S.E_sc + 3 * (8 * sc + comp), e, S.err);
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
// v added into the accumulators of the three entries of node i
__device__ inline void acc_add3(acc_t* a, int i, d3 v, int* err) {
  acc_add(a + 9 * (size_t)i, v.x, err);
  acc_add(a + 9 * (size_t)i + 3, v.y, err);
  acc_add(a + 9 * (size_t)i + 6, v.z, err);
}


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
  v = (threadIdx.x < nw) ? shm[threadIdx.x] : -INFINITY;  // lanes without a warp must not raise the maximum
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


}  // namespace ipc
