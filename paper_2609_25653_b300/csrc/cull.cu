// Contact candidate culling and continuous collision detection (§III-C.1:
// barrier potentials together with continuous collision detection).
//
// Active set: every (surface vertex, surface triangle) and (surface edge,
// surface edge) pair with squared distance below dhat^2, after the exclusion
// rules (shared vertex; both primitives on one rigid or kinematic body; both
// kinematic).  CCD: the additive-CCD time of impact of every pair whose
// swept boxes over [x, x + p] overlap; the step bound is their minimum.
//
// This file is compiled with -fmad=false: the classification and the
// squared distance that decide membership (s < dhat^2) round operation by
// operation as written, so the active set is exactly reproducible.
#include <algorithm>
#include "bvh.cuh"
#include "common.cuh"
#include "dist.cuh"
#include "kernels.h"

namespace ipc {

__device__ inline bool excluded(const DevScene& S, const int* va, int na, const int* vb, int nb) {
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j)
      if (va[i] == vb[j]) return true;
  int ba = S.vbody[va[0]], bb = S.vbody[vb[0]];
  if (S.body_scene[ba] != S.body_scene[bb]) return true;  // independent scenes of a batch
  int ka = S.bkind[ba], kb = S.bkind[bb];
  if (ba == bb && ka != VK_FEM) return true;
  if (ka == VK_KIN && kb == VK_KIN) return true;
  return false;
}

// counters stop near 2^30 so that they never wrap; the host reports the overflow
constexpr int COUNT_CEILING = 1 << 30;

__device__ inline void emit(int* rec, double* rec_s, int* count, int cap, int kind, int a, int b, int type,
                            const int* ids, double s) {
  if (*(volatile int*)count >= COUNT_CEILING) return;
  int slot = atomicAdd(count, 1);
  if (slot < cap) {
    int* r = rec + 8 * (size_t)slot;
    r[0] = kind; r[1] = a; r[2] = b; r[3] = type;
    r[4] = ids[0]; r[5] = ids[1]; r[6] = ids[2]; r[7] = ids[3];
    if (rec_s) rec_s[slot] = s;
  }
}

// Point-triangle pairs: thread per (surface vertex i, triangle t)
__global__ void k_cull_pt_brute(DevScene S, const double* __restrict__ xv, double sh, int* rec, double* rec_s,
                                int* count, int cap) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)S.nsv * S.ntri;
  if (idx >= total) return;
  int i = (int)(idx / S.ntri), t = (int)(idx % S.ntri);
  int p = S.sv[i];
  int3 tv = S.tris[t];
  int tvv[3] = {tv.x, tv.y, tv.z};
  if (excluded(S, &p, 1, tvv, 3)) return;
  int ids[4] = {p, tv.x, tv.y, tv.z};
  d3 x[4] = {ld3(xv, p), ld3(xv, tv.x), ld3(xv, tv.y), ld3(xv, tv.z)};
  double s, w[4];
  int type = pt_classify(x, s, w);
  if (s < sh) emit(rec, rec_s, count, cap, 0, i, t, type, ids, s);
}

// Edge-edge pairs: thread per (edge a, edge b), a < b
__global__ void k_cull_ee_brute(DevScene S, const double* __restrict__ xv, double sh, int* rec, double* rec_s,
                                int* count, int cap) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)S.nedge * S.nedge;
  if (idx >= total) return;
  int ea = (int)(idx / S.nedge), eb = (int)(idx % S.nedge);
  if (eb <= ea) return;
  int2 A = S.edges[ea], B = S.edges[eb];
  int va[2] = {A.x, A.y}, vb[2] = {B.x, B.y};
  if (excluded(S, va, 2, vb, 2)) return;
  int ids[4] = {A.x, A.y, B.x, B.y};
  d3 x[4] = {ld3(xv, A.x), ld3(xv, A.y), ld3(xv, B.x), ld3(xv, B.y)};
  double s, w[4];
  int type = ee_classify(x, s, w);
  if (s < sh) emit(rec, rec_s, count, cap, 1, ea, eb, type, ids, s);
}

// ---------------------------------------------------------------------------
// additive CCD (Li et al., "Codimensional Incremental Potential Contact", 2021)
// ---------------------------------------------------------------------------
// The distance of the stencil can shrink at most at rate lp (the two
// primitives' largest speeds relative to the stencil mean), so advancing by
// (1 - s) d0 / lp, then by 0.9 d / lp, never passes a contact.  Stops before
// the distance falls below s d0; returns tmax if that does not happen.
__device__ double accd(int kind, const d3* x0, const d3* p0, double s_frac, double tmax, int max_iter) {
  d3 pbar = mk(0.0, 0.0, 0.0);
  for (int k = 0; k < 4; ++k) pbar = pbar + 0.25 * p0[k];
  d3 p[4];
  double nrm[4];
  for (int k = 0; k < 4; ++k) {
    p[k] = p0[k] - pbar;
    nrm[k] = sqrt(dot(p[k], p[k]));
  }
  double lp = (kind == 0) ? nrm[0] + fmax(nrm[1], fmax(nrm[2], nrm[3])) : fmax(nrm[0], nrm[1]) + fmax(nrm[2], nrm[3]);
  if (lp == 0.0) return tmax;
  // A cheap lower bound of the distance (point or edge against the other primitive's bounding
  // sphere): when even it allows a first advance (1 - s) d0 / lp past tmax, the result is tmax.
  // The margin keeps the bound's own rounding from deciding a borderline pair.
  {
    d3 ca, cb;
    double ra, rb;
    if (kind == 0) {
      ca = x0[0];
      ra = 0.0;
      cb = (1.0 / 3.0) * (x0[1] + x0[2] + x0[3]);
      rb = 0.0;
      for (int k = 1; k < 4; ++k) { d3 e = x0[k] - cb; rb = fmax(rb, sqrt(dot(e, e))); }
    } else {
      ca = 0.5 * (x0[0] + x0[1]);
      cb = 0.5 * (x0[2] + x0[3]);
      d3 ea = x0[0] - ca, eb = x0[2] - cb;
      ra = sqrt(dot(ea, ea));
      rb = sqrt(dot(eb, eb));
    }
    d3 dc = ca - cb;
    const double lb = sqrt(dot(dc, dc)) - ra - rb;
    if (lb > 0.0 && (1.0 - s_frac) * lb >= tmax * lp * (1.0 + 1e-9)) return tmax;
  }
  double d0 = sqrt(pair_s(kind, x0));
  double target = s_frac * d0;
  double t = 0.0, tl = (1.0 - s_frac) * d0 / lp;
  // the distance at the first advance only sets the next step: not needed when it already reaches tmax
  if (tl >= tmax) return tmax;
  d3 xt[4];
  for (int it = 0; it < max_iter; ++it) {
    double tn = t + tl;
    for (int k = 0; k < 4; ++k) xt[k] = mk(x0[k].x + tn * p[k].x, x0[k].y + tn * p[k].y, x0[k].z + tn * p[k].z);
    double d = sqrt(pair_s(kind, xt));
    if (d < target && it > 0) return t;
    t = tn;
    if (t >= tmax) return tmax;
    tl = 0.9 * d / lp;
  }
  return t;
}

// Upper bound handed to ACCD by the traversal kernels.  Only a time of impact
// below the running minimum of the pair's scene can change that minimum, and
// ACCD with a smaller bound tmax returns min(its result with bound 1, tmax)
// from the same arithmetic (it stops once its time reaches tmax, and its
// early-outs only fire when the result would be at least tmax), so the
// minimum over the pairs is unchanged while more pairs stop early.
__device__ inline double ccd_tmax(const DevScene& S, const unsigned long long* alpha_bits, int sc, double amin) {
  const unsigned long long* src = S.alpha_sc ? S.alpha_sc + sc : alpha_bits;
  const double cur = __longlong_as_double((long long)*(const volatile unsigned long long*)src);
  return fmin(amin, fmin(cur, 1.0));
}

__device__ inline void swept(const double* xv, const double* pv, int v, d3& lo, d3& hi) {
  d3 a = ld3(xv, v), p = ld3(pv, v);
  d3 b = a + p;
  lo = mk(fmin(lo.x, fmin(a.x, b.x)), fmin(lo.y, fmin(a.y, b.y)), fmin(lo.z, fmin(a.z, b.z)));
  hi = mk(fmax(hi.x, fmax(a.x, b.x)), fmax(hi.y, fmax(a.y, b.y)), fmax(hi.z, fmax(a.z, b.z)));
}
__device__ inline bool overlap(d3 la, d3 ha, d3 lb, d3 hb) {
  return !(la.x > hb.x || lb.x > ha.x || la.y > hb.y || lb.y > ha.y || la.z > hb.z || lb.z > ha.z);
}

__global__ void k_ccd_pt_brute(DevScene S, const double* __restrict__ xv, const double* __restrict__ pv, double s_frac,
                               int max_iter, unsigned long long* alpha_bits, int* n_cand) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)S.nsv * S.ntri;
  if (idx >= total) return;
  int i = (int)(idx / S.ntri), t = (int)(idx % S.ntri);
  int p = S.sv[i];
  int3 tv = S.tris[t];
  int tvv[3] = {tv.x, tv.y, tv.z};
  if (excluded(S, &p, 1, tvv, 3)) return;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  d3 la = mk(inf, inf, inf), ha = mk(-inf, -inf, -inf), lb = la, hb = ha;
  swept(xv, pv, p, la, ha);
  swept(xv, pv, tv.x, lb, hb);
  swept(xv, pv, tv.y, lb, hb);
  swept(xv, pv, tv.z, lb, hb);
  if (!overlap(la, ha, lb, hb)) return;
  int ids[4] = {p, tv.x, tv.y, tv.z};
  d3 x[4], pp[4];
  for (int k = 0; k < 4; ++k) { x[k] = ld3(xv, ids[k]); pp[k] = ld3(pv, ids[k]); }
  atomicAdd(n_cand, 1);
  double toi = accd(0, x, pp, s_frac, 1.0, max_iter);
  if (toi < 1.0) {
    atomicMin(alpha_bits, dbits(toi));
    if (S.alpha_sc) atomicMin(S.alpha_sc + scene_of_vertex(S, p), dbits(toi));
  }
}

__global__ void k_ccd_ee_brute(DevScene S, const double* __restrict__ xv, const double* __restrict__ pv, double s_frac,
                               int max_iter, unsigned long long* alpha_bits, int* n_cand) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)S.nedge * S.nedge;
  if (idx >= total) return;
  int ea = (int)(idx / S.nedge), eb = (int)(idx % S.nedge);
  if (eb <= ea) return;
  int2 A = S.edges[ea], B = S.edges[eb];
  int va[2] = {A.x, A.y}, vb[2] = {B.x, B.y};
  if (excluded(S, va, 2, vb, 2)) return;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  d3 la = mk(inf, inf, inf), ha = mk(-inf, -inf, -inf), lb = la, hb = ha;
  swept(xv, pv, A.x, la, ha);
  swept(xv, pv, A.y, la, ha);
  swept(xv, pv, B.x, lb, hb);
  swept(xv, pv, B.y, lb, hb);
  if (!overlap(la, ha, lb, hb)) return;
  int ids[4] = {A.x, A.y, B.x, B.y};
  d3 x[4], pp[4];
  for (int k = 0; k < 4; ++k) { x[k] = ld3(xv, ids[k]); pp[k] = ld3(pv, ids[k]); }
  atomicAdd(n_cand, 1);
  double toi = accd(1, x, pp, s_frac, 1.0, max_iter);
  if (toi < 1.0) {
    atomicMin(alpha_bits, dbits(toi));
    if (S.alpha_sc) atomicMin(S.alpha_sc + scene_of_vertex(S, ids[0]), dbits(toi));
  }
}

// ---------------------------------------------------------------------------
// LBVH queries: the same exact tests as above, on the leaves whose boxes overlap
// ---------------------------------------------------------------------------
constexpr int STACK = 64;

struct TreeView {
  int n;
  const int* prim;
  const int* left;
  const int* right;
  const float* box;
};
__host__ inline TreeView view(const Bvh& B) { return TreeView{B.n, B.prim, B.left, B.right, B.box}; }

// Visit every leaf whose box overlaps q (in the outward-rounded FP32 boxes of
// the tree, a superset of the exact overlaps); f(primitive) per leaf.  Returns
// false on stack overflow.
template <typename F>
__device__ inline bool traverse(const TreeView& T, const double* q64, F f) {
  if (T.n <= 0) return true;
  float q[6];
  box_outward(q64, q);
  int stack[STACK];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    int node = stack[--sp];
    if (!box_overlap(T.box + 6 * (size_t)node, q)) continue;
    if (node >= T.n - 1) {
      f(T.prim[node - (T.n - 1)]);
    } else {
      if (sp + 2 > STACK) return false;
      stack[sp++] = T.right[node];
      stack[sp++] = T.left[node];
    }
  }
  return true;
}

// Active point-triangle pairs: thread per surface vertex; the triangle leaves carry boxes widened by >= dhat.
__global__ void k_cull_pt_bvh(DevScene S, const double* __restrict__ xv, double sh, TreeView T, int* rec, double* rec_s,
                              int* count, int cap, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.nsv) return;
  int p = S.sv[i];
  d3 xp = ld3(xv, p);
  double q[6] = {xp.x, xp.y, xp.z, xp.x, xp.y, xp.z};
  bool ok = traverse(T, q, [&](int t) {
    int3 tv = S.tris[t];
    int tvv[3] = {tv.x, tv.y, tv.z};
    if (excluded(S, &p, 1, tvv, 3)) return;
    int ids[4] = {p, tv.x, tv.y, tv.z};
    d3 x[4] = {xp, ld3(xv, tv.x), ld3(xv, tv.y), ld3(xv, tv.z)};
    double s, w[4];
    int type = pt_classify(x, s, w);
    if (s < sh) emit(rec, rec_s, count, cap, 0, i, t, type, ids, s);
  });
  if (!ok) atomicOr(err, ERRF_BVH);
}

// Active edge-edge pairs: thread per edge a, pairs with b > a; edge leaves widened by >= dhat.
__global__ void k_cull_ee_bvh(DevScene S, const double* __restrict__ xv, double sh, TreeView T, int* rec, double* rec_s,
                              int* count, int cap, int* err) {
  int ea = blockIdx.x * blockDim.x + threadIdx.x;
  if (ea >= S.nedge) return;
  int2 A = S.edges[ea];
  // edges are sorted by vertex id and kinematic vertices come last: every edge after a
  // kinematic edge is kinematic, so this query could only meet excluded pairs
  if (S.vkind[A.x] == VK_KIN) return;
  d3 a0 = ld3(xv, A.x), a1 = ld3(xv, A.y);
  double q[6] = {fmin(a0.x, a1.x), fmin(a0.y, a1.y), fmin(a0.z, a1.z), fmax(a0.x, a1.x), fmax(a0.y, a1.y), fmax(a0.z, a1.z)};
  bool ok = traverse(T, q, [&](int eb) {
    if (eb <= ea) return;
    int2 B = S.edges[eb];
    int va[2] = {A.x, A.y}, vb[2] = {B.x, B.y};
    if (excluded(S, va, 2, vb, 2)) return;
    int ids[4] = {A.x, A.y, B.x, B.y};
    d3 x[4] = {a0, a1, ld3(xv, B.x), ld3(xv, B.y)};
    double s, w[4];
    int type = ee_classify(x, s, w);
    if (s < sh) emit(rec, rec_s, count, cap, 1, ea, eb, type, ids, s);
  });
  if (!ok) atomicOr(err, ERRF_BVH);
}

// CCD candidates: leaves carry swept boxes over [x, x + p]; the query is the swept box of the point / edge.
__global__ void k_ccd_pt_bvh(DevScene S, const double* __restrict__ xv, const double* __restrict__ pv, double s_frac,
                             int max_iter, TreeView T, unsigned long long* alpha_bits, int* n_cand, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.nsv) return;
  int p = S.sv[i];
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  d3 la = mk(inf, inf, inf), ha = mk(-inf, -inf, -inf);
  swept(xv, pv, p, la, ha);
  double q[6] = {la.x, la.y, la.z, ha.x, ha.y, ha.z};
  double amin = 1.0;
  const int sc = S.alpha_sc ? scene_of_vertex(S, p) : 0;
  int nc = 0;
  bool ok = traverse(T, q, [&](int t) {
    int3 tv = S.tris[t];
    int tvv[3] = {tv.x, tv.y, tv.z};
    if (excluded(S, &p, 1, tvv, 3)) return;
    // the exact FP64 swept-box test (the tree's FP32 boxes are a conservative superset)
    d3 lb = mk(inf, inf, inf), hb = mk(-inf, -inf, -inf);
    swept(xv, pv, tv.x, lb, hb);
    swept(xv, pv, tv.y, lb, hb);
    swept(xv, pv, tv.z, lb, hb);
    if (!overlap(la, ha, lb, hb)) return;
    int ids[4] = {p, tv.x, tv.y, tv.z};
    d3 x[4], pp[4];
    for (int k = 0; k < 4; ++k) { x[k] = ld3(xv, ids[k]); pp[k] = ld3(pv, ids[k]); }
    ++nc;
    amin = fmin(amin, accd(0, x, pp, s_frac, ccd_tmax(S, alpha_bits, sc, amin), max_iter));
  });
  if (!ok) atomicOr(err, ERRF_BVH);
  if (nc) atomicAdd(n_cand, nc);
  if (amin < 1.0) {
    atomicMin(alpha_bits, dbits(amin));
    if (S.alpha_sc) atomicMin(S.alpha_sc + scene_of_vertex(S, p), dbits(amin));
  }
}

__global__ void k_ccd_ee_bvh(DevScene S, const double* __restrict__ xv, const double* __restrict__ pv, double s_frac,
                             int max_iter, TreeView T, unsigned long long* alpha_bits, int* n_cand, int* err) {
  int ea = blockIdx.x * blockDim.x + threadIdx.x;
  if (ea >= S.nedge) return;
  int2 A = S.edges[ea];
  if (S.vkind[A.x] == VK_KIN) return;  // only kinematic edges follow: all pairs excluded
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  d3 la = mk(inf, inf, inf), ha = mk(-inf, -inf, -inf);
  swept(xv, pv, A.x, la, ha);
  swept(xv, pv, A.y, la, ha);
  double q[6] = {la.x, la.y, la.z, ha.x, ha.y, ha.z};
  double amin = 1.0;
  const int sc = S.alpha_sc ? scene_of_vertex(S, A.x) : 0;
  int nc = 0;
  bool ok = traverse(T, q, [&](int eb) {
    if (eb <= ea) return;
    int2 B = S.edges[eb];
    int va[2] = {A.x, A.y}, vb[2] = {B.x, B.y};
    if (excluded(S, va, 2, vb, 2)) return;
    d3 lb = mk(inf, inf, inf), hb = mk(-inf, -inf, -inf);
    swept(xv, pv, B.x, lb, hb);
    swept(xv, pv, B.y, lb, hb);
    if (!overlap(la, ha, lb, hb)) return;
    int ids[4] = {A.x, A.y, B.x, B.y};
    d3 x[4], pp[4];
    for (int k = 0; k < 4; ++k) { x[k] = ld3(xv, ids[k]); pp[k] = ld3(pv, ids[k]); }
    ++nc;
    amin = fmin(amin, accd(1, x, pp, s_frac, ccd_tmax(S, alpha_bits, sc, amin), max_iter));
  });
  if (!ok) atomicOr(err, ERRF_BVH);
  if (nc) atomicAdd(n_cand, nc);
  if (amin < 1.0) {
    atomicMin(alpha_bits, dbits(amin));
    if (S.alpha_sc) atomicMin(S.alpha_sc + scene_of_vertex(S, A.x), dbits(amin));
  }
}

// ---------------------------------------------------------------------------
// one sweep per Newton iteration: CCD bound and contact candidates together
// ---------------------------------------------------------------------------
// Leaves carry swept boxes over [x, x + p] widened by pad (>= dhat).  Every
// non-excluded pair whose query box (the unwidened swept box of the point or
// edge) overlaps a leaf is a candidate: it contains every pair that comes
// within dhat anywhere on the segment, so the active sets along the line
// search and at the next iterate are exactly the candidates with s < dhat^2.
// Candidates whose unwidened swept boxes overlap also get the ACCD time of
// impact, which reproduces the CCD of the plain sweep.
__device__ inline void emit_cand(int* cand, int* n_cand, int ccap, int kind, int a, int b, const int* ids) {
  if (*(volatile int*)n_cand >= COUNT_CEILING) return;
  int slot = atomicAdd(n_cand, 1);
  if (slot < ccap) {
    int* r = cand + 8 * (size_t)slot;
    r[0] = kind; r[1] = a; r[2] = b; r[3] = -1;
    r[4] = ids[0]; r[5] = ids[1]; r[6] = ids[2]; r[7] = ids[3];
  }
}

// Sweep traversal: every (point, triangle) and (edge, edge) pair whose padded
// swept boxes overlap becomes a candidate (the line search and the next
// iterate take their active pairs from this list).  The CCD of the
// candidates runs afterwards in k_ccd_cand: evaluating it inside the
// traversal left a few lanes of each warp doing FP64 work while the others
// walked the tree.
__global__ void k_sweep_pt_bvh(DevScene S, const double* __restrict__ xv, const double* __restrict__ pv, TreeView T,
                               int* cand, int* n_cand, int ccap, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.nsv) return;
  int p = S.sv[i];
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  d3 la = mk(inf, inf, inf), ha = mk(-inf, -inf, -inf);
  swept(xv, pv, p, la, ha);
  double q[6] = {la.x, la.y, la.z, ha.x, ha.y, ha.z};
  bool ok = traverse(T, q, [&](int t) {
    int3 tv = S.tris[t];
    int tvv[3] = {tv.x, tv.y, tv.z};
    if (excluded(S, &p, 1, tvv, 3)) return;
    int ids[4] = {p, tv.x, tv.y, tv.z};
    emit_cand(cand, n_cand, ccap, 0, i, t, ids);
  });
  if (!ok) atomicOr(err, ERRF_BVH);
}

__global__ void k_sweep_ee_bvh(DevScene S, const double* __restrict__ xv, const double* __restrict__ pv, TreeView T,
                               int* cand, int* n_cand, int ccap, int* err) {
  int ea = blockIdx.x * blockDim.x + threadIdx.x;
  if (ea >= S.nedge) return;
  int2 A = S.edges[ea];
  if (S.vkind[A.x] == VK_KIN) return;  // only kinematic edges follow: all pairs excluded
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  d3 la = mk(inf, inf, inf), ha = mk(-inf, -inf, -inf);
  swept(xv, pv, A.x, la, ha);
  swept(xv, pv, A.y, la, ha);
  double q[6] = {la.x, la.y, la.z, ha.x, ha.y, ha.z};
  bool ok = traverse(T, q, [&](int eb) {
    if (eb <= ea) return;
    int2 B = S.edges[eb];
    int va[2] = {A.x, A.y}, vb[2] = {B.x, B.y};
    if (excluded(S, va, 2, vb, 2)) return;
    int ids[4] = {A.x, A.y, B.x, B.y};
    emit_cand(cand, n_cand, ccap, 1, ea, eb, ids);
  });
  if (!ok) atomicOr(err, ERRF_BVH);
}

// CCD of the sweep's candidates, one candidate per thread: the exact FP64
// swept-box test (the tree's boxes are padded and FP32), then ACCD bounded by
// the running minimum of the pair's scene; a result below that bound lowers
// the scene's and the global step bound.  n_ccd counts the ACCD evaluations.
// Reads at most ccap candidates: when more were found the host enlarges the
// list and repeats the Newton iteration before it uses the bound.
__global__ void __launch_bounds__(128) k_ccd_cand(DevScene S, const double* __restrict__ xv,
                                                  const double* __restrict__ pv, double s_frac, int max_iter,
                                                  const int* __restrict__ cand, const int* __restrict__ n_cand,
                                                  int ccap, unsigned long long* alpha_bits, int* n_ccd) {
  const int n = min(*n_cand, ccap);
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  int nc = 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const int* r = cand + 8 * (size_t)c;
    const int kind = r[0];
    const int ids[4] = {r[4], r[5], r[6], r[7]};
    const int na = kind == 0 ? 1 : 2;  // vertices of the first primitive
    d3 la = mk(inf, inf, inf), ha = mk(-inf, -inf, -inf), lb = la, hb = ha;
    for (int k = 0; k < 4; ++k) {
      if (k < na) swept(xv, pv, ids[k], la, ha);
      else swept(xv, pv, ids[k], lb, hb);
    }
    if (!overlap(la, ha, lb, hb)) continue;
    d3 x[4], pp[4];
    for (int k = 0; k < 4; ++k) { x[k] = ld3(xv, ids[k]); pp[k] = ld3(pv, ids[k]); }
    ++nc;
    const int sc = S.alpha_sc ? scene_of_vertex(S, ids[0]) : 0;
    const double tmax = ccd_tmax(S, alpha_bits, sc, 1.0);
    const double t = accd(kind, x, pp, s_frac, tmax, max_iter);
    if (t < tmax) {
      atomicMin(alpha_bits, dbits(t));
      if (S.alpha_sc) atomicMin(S.alpha_sc + sc, dbits(t));
    }
  }
  nc = __reduce_add_sync(0xffffffffu, nc);
  if ((threadIdx.x & 31) == 0 && nc) atomicAdd(n_ccd, nc);
}

// Active pairs among the candidates: the exact classification and s < dhat^2 at xv.
__global__ void k_filter_active(DevScene S, const double* __restrict__ xv, double sh, const int* __restrict__ cand,
                                const int* __restrict__ n_cand, int ccap, int* rec, double* rec_s, int* count, int cap) {
  int n = min(*n_cand, ccap);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const int* r = cand + 8 * (size_t)c;
    int kind = r[0];
    int ids[4] = {r[4], r[5], r[6], r[7]};
    d3 x[4] = {ld3(xv, ids[0]), ld3(xv, ids[1]), ld3(xv, ids[2]), ld3(xv, ids[3])};
    double s, w[4];
    int type = kind == 0 ? pt_classify(x, s, w) : ee_classify(x, s, w);
    if (s < sh) emit(rec, rec_s, count, cap, kind, r[1], r[2], type, ids, s);
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
void launch_cull_brute(cudaStream_t st, const DevScene& S, const double* xv, double sh, int* rec, double* rec_s,
                       int* count, int cap) {
  long long npt = (long long)S.nsv * S.ntri, nee = (long long)S.nedge * S.nedge;
  if (npt) { k_cull_pt_brute<<<(unsigned)((npt + 255) / 256), 256, 0, st>>>(S, xv, sh, rec, rec_s, count, cap); count_launch(); }
  if (nee) { k_cull_ee_brute<<<(unsigned)((nee + 255) / 256), 256, 0, st>>>(S, xv, sh, rec, rec_s, count, cap); count_launch(); }
}

void launch_ccd_brute(cudaStream_t st, const DevScene& S, const double* xv, const double* pv, double s_frac,
                      int max_iter, unsigned long long* alpha_bits, int* n_cand) {
  long long npt = (long long)S.nsv * S.ntri, nee = (long long)S.nedge * S.nedge;
  if (npt) { k_ccd_pt_brute<<<(unsigned)((npt + 255) / 256), 256, 0, st>>>(S, xv, pv, s_frac, max_iter, alpha_bits, n_cand); count_launch(); }
  if (nee) { k_ccd_ee_brute<<<(unsigned)((nee + 255) / 256), 256, 0, st>>>(S, xv, pv, s_frac, max_iter, alpha_bits, n_cand); count_launch(); }
}

}  // namespace ipc

namespace ipc {

// Active set through the trees: refit both trees on boxes widened by pad, then query.
void launch_cull_bvh(cudaStream_t st, const DevScene& S, const double* xv, double sh, double pad, Bvh& tri, Bvh& edge,
                     int* rec, double* rec_s, int* count, int cap, int* err) {
  bvh_leaf_boxes(st, tri, (const int*)S.tris, 3, xv, nullptr, pad);
  bvh_refit(st, tri);
  bvh_leaf_boxes(st, edge, (const int*)S.edges, 2, xv, nullptr, pad);
  bvh_refit(st, edge);
  if (S.nsv) { k_cull_pt_bvh<<<(S.nsv + 127) / 128, 128, 0, st>>>(S, xv, sh, view(tri), rec, rec_s, count, cap, err); count_launch(); }
  if (S.nedge) { k_cull_ee_bvh<<<(S.nedge + 127) / 128, 128, 0, st>>>(S, xv, sh, view(edge), rec, rec_s, count, cap, err); count_launch(); }
}

void launch_ccd_bvh(cudaStream_t st, const DevScene& S, const double* xv, const double* pv, double s_frac, int max_iter,
                    Bvh& tri, Bvh& edge, unsigned long long* alpha_bits, int* n_cand, int* err) {
  bvh_leaf_boxes(st, tri, (const int*)S.tris, 3, xv, pv, 0.0);
  bvh_refit(st, tri);
  bvh_leaf_boxes(st, edge, (const int*)S.edges, 2, xv, pv, 0.0);
  bvh_refit(st, edge);
  if (S.nsv) { k_ccd_pt_bvh<<<(S.nsv + 127) / 128, 128, 0, st>>>(S, xv, pv, s_frac, max_iter, view(tri), alpha_bits, n_cand, err); count_launch(); }
  if (S.nedge) { k_ccd_ee_bvh<<<(S.nedge + 127) / 128, 128, 0, st>>>(S, xv, pv, s_frac, max_iter, view(edge), alpha_bits, n_cand, err); count_launch(); }
}

// Rebuild both trees (Morton sort + hierarchy) on boxes at xv widened by pad.
void bvh_rebuild(cudaStream_t st, const DevScene& S, const double* xv, double pad, Bvh& tri, Bvh& edge) {
  bvh_leaf_boxes(st, tri, (const int*)S.tris, 3, xv, nullptr, pad);
  bvh_build(st, tri);
  bvh_leaf_boxes(st, edge, (const int*)S.edges, 2, xv, nullptr, pad);
  bvh_build(st, edge);
}

}  // namespace ipc

namespace ipc {

void launch_sweep_bvh(cudaStream_t st, const DevScene& S, const double* xv, const double* pv, double pad, double s_frac,
                      int max_iter, Bvh& tri, Bvh& edge, int* cand, int* n_cand, int ccap,
                      unsigned long long* alpha_bits, int* n_ccd, int* err) {
  bvh_leaf_boxes(st, tri, (const int*)S.tris, 3, xv, pv, pad);
  bvh_refit(st, tri);
  bvh_leaf_boxes(st, edge, (const int*)S.edges, 2, xv, pv, pad);
  bvh_refit(st, edge);
  if (S.nsv) { k_sweep_pt_bvh<<<(S.nsv + 127) / 128, 128, 0, st>>>(S, xv, pv, view(tri), cand, n_cand, ccap, err); count_launch(); }
  if (S.nedge) { k_sweep_ee_bvh<<<(S.nedge + 127) / 128, 128, 0, st>>>(S, xv, pv, view(edge), cand, n_cand, ccap, err); count_launch(); }
  if (ccap > 0) {
    const int grid = stride_grid(ccap, 128, 16);
    k_ccd_cand<<<grid, 128, 0, st>>>(S, xv, pv, s_frac, max_iter, cand, n_cand, ccap, alpha_bits, n_ccd);
    count_launch();
  }
}

void launch_filter_active(cudaStream_t st, int grid, const DevScene& S, const double* xv, double sh, const int* cand,
                          const int* n_cand, int ccap, int* rec, double* rec_s, int* count, int cap) {
  k_filter_active<<<grid, 128, 0, st>>>(S, xv, sh, cand, n_cand, ccap, rec, rec_s, count, cap);
  count_launch();
}

}  // namespace ipc
