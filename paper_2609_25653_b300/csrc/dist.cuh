// Point-triangle and edge-edge squared distances on the device.
//
// Distance types (closest-point configuration):
//   point-triangle (p, t0, t1, t2): 0,1,2 point-point with t0,t1,t2;
//     3,4,5 point-edge (t0t1), (t1t2), (t2t0); 6 point-plane.
//   edge-edge (a0, a1, b0, b1): 0..3 point-point (a0b0, a0b1, a1b0, a1b1);
//     4,5 b0 / b1 against edge a; 6,7 a0 / a1 against edge b; 8 line-line.
// The classification takes the unconstrained closest points when they lie
// inside both primitives and otherwise the nearest boundary configuration.
//
// The culling translation unit is compiled with -fmad=false so that the
// squared distance that decides membership of the active set (s < dhat^2)
// rounds exactly as the plain definition written here, operation by
// operation.
#pragma once
#include "common.cuh"

namespace ipc {

__device__ inline double s_pp(d3 a, d3 b) {
  d3 d = a - b;
  return dot(d, d);
}
__device__ inline double s_pe(d3 p, d3 e0, d3 e1) {
  d3 r = p - e0, e = e1 - e0;
  double c = dot(r, e), q = dot(e, e);
  return dot(r, r) - c * c / q;
}
__device__ inline double s_plane(d3 v, d3 a, d3 b) {
  d3 n = cross(a, b);
  double c = dot(v, n), q = dot(n, n);
  return c * c / q;
}
__device__ inline double seg_t(d3 p, d3 e0, d3 e1) {
  d3 r = p - e0, e = e1 - e0;
  double t = dot(r, e) / dot(e, e);
  return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
}

__device__ inline double pt_type_s(const d3* x, int type) {
  if (type <= 2) return s_pp(x[0], x[1 + type]);
  if (type <= 5) return s_pe(x[0], x[1 + (type - 3)], x[1 + (type - 2) % 3]);
  return s_plane(x[0] - x[1], x[2] - x[1], x[3] - x[1]);
}

__device__ inline double ee_type_s(const d3* x, int type) {
  switch (type) {
    case 0: return s_pp(x[0], x[2]);
    case 1: return s_pp(x[0], x[3]);
    case 2: return s_pp(x[1], x[2]);
    case 3: return s_pp(x[1], x[3]);
    case 4: return s_pe(x[2], x[0], x[1]);
    case 5: return s_pe(x[3], x[0], x[1]);
    case 6: return s_pe(x[0], x[2], x[3]);
    case 7: return s_pe(x[1], x[2], x[3]);
    default: return s_plane(x[0] - x[2], x[1] - x[0], x[3] - x[2]);
  }
}

// Returns the type; s = that type's squared distance; w = closest-point
// weights with sum_k w_k x_k = (point on the first primitive) - (point on the second).
__device__ inline int pt_classify(const d3* x, double& s, double* w) {
  d3 a = x[2] - x[1], b = x[3] - x[1], v = x[0] - x[1];
  double aa = dot(a, a), ab = dot(a, b), bb = dot(b, b), av = dot(a, v), bv = dot(b, v);
  double det = aa * bb - ab * ab;
  double b1 = (bb * av - ab * bv) / det, b2 = (aa * bv - ab * av) / det;
  if (b1 > 0.0 && b2 > 0.0 && b1 + b2 < 1.0) {
    s = pt_type_s(x, 6);
    w[0] = 1.0; w[1] = -(1.0 - b1 - b2); w[2] = -b1; w[3] = -b2;
    return 6;
  }
  int best = -1;
  double best_s = 0.0, best_t = 0.0;
  for (int k = 0; k < 3; ++k) {
    double t = seg_t(x[0], x[1 + k], x[1 + (k + 1) % 3]);
    int type = (t == 0.0) ? k : (t == 1.0 ? (k + 1) % 3 : 3 + k);
    double sk = pt_type_s(x, type);
    if (best < 0 || sk < best_s) { best = type; best_s = sk; best_t = t; }
  }
  s = best_s;
  w[0] = 1.0; w[1] = w[2] = w[3] = 0.0;
  if (best <= 2) w[1 + best] = -1.0;
  else {
    int k = best - 3;
    w[1 + k] = -(1.0 - best_t);
    w[1 + (k + 1) % 3] = -best_t;
  }
  return best;
}

__device__ inline int ee_classify(const d3* x, double& s, double* w) {
  d3 u = x[1] - x[0], v = x[3] - x[2], r = x[0] - x[2];
  double uu = dot(u, u), uv = dot(u, v), vv = dot(v, v), ur = dot(u, r), vr = dot(v, r);
  double D = uu * vv - uv * uv;
  if (D > 1e-12 * uu * vv) {
    double sa = (uv * vr - vv * ur) / D, tb = (uu * vr - uv * ur) / D;
    if (sa > 0.0 && sa < 1.0 && tb > 0.0 && tb < 1.0) {
      s = ee_type_s(x, 8);
      w[0] = 1.0 - sa; w[1] = sa; w[2] = -(1.0 - tb); w[3] = -tb;
      return 8;
    }
  }
  // an endpoint against the other segment: (point slot, segment slots)
  const int cpt[4] = {2, 3, 0, 1}, ce0[4] = {0, 0, 2, 2}, ce1[4] = {1, 1, 3, 3};
  int best = -1, best_c = 0;
  double best_s = 0.0, best_t = 0.0;
  for (int c = 0; c < 4; ++c) {
    double t = seg_t(x[cpt[c]], x[ce0[c]], x[ce1[c]]);
    int type;
    if (t > 0.0 && t < 1.0) type = 4 + c;
    else {
      int other = (t == 0.0) ? ce0[c] : ce1[c];
      int ia = cpt[c] < 2 ? cpt[c] : other;
      int ib = cpt[c] < 2 ? other : cpt[c];
      type = 2 * ia + (ib - 2);
    }
    double sc = ee_type_s(x, type);
    if (best < 0 || sc < best_s) { best = type; best_s = sc; best_t = t; best_c = c; }
  }
  s = best_s;
  w[0] = w[1] = w[2] = w[3] = 0.0;
  if (best <= 3) {
    w[best / 2] = 1.0;
    w[2 + best % 2] = -1.0;
  } else {
    double sg = cpt[best_c] < 2 ? 1.0 : -1.0;
    w[cpt[best_c]] = sg;
    w[ce0[best_c]] = -sg * (1.0 - best_t);
    w[ce1[best_c]] = -sg * best_t;
  }
  return best;
}

__device__ inline double pair_s(int kind, const d3* x) {
  double s, w[4];
  if (kind == 0) pt_classify(x, s, w);
  else ee_classify(x, s, w);
  return s;
}

// ---------------------------------------------------------------------------
// derivatives of the squared distance of a given type (12 DOFs, stencil order)
// ---------------------------------------------------------------------------
// Each type is a function of up to three "difference" variables u_m = sum_k
// C[m][k] x_k.  First and second derivatives are taken in those variables
// and mapped back: g_k = sum_m C[m][k] g_m, H_kl = sum_mn C[m][k] C[n][l] H_mn.

struct Red {
  int nv;
  double C[3][4];
  d3 g[3];
  double H[3][3][9];  // H[m][n] 3x3 block, row-major
};

__device__ inline void skew9(d3 w, double* M) {
  M[0] = 0; M[1] = -w.z; M[2] = w.y;
  M[3] = w.z; M[4] = 0; M[5] = -w.x;
  M[6] = -w.y; M[7] = w.x; M[8] = 0;
}
__device__ inline void mm3(const double* A, const double* B, double* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

__device__ inline void red_pp(Red& R, d3 d) {
  R.nv = 1;
  R.g[0] = 2.0 * d;
  for (int q = 0; q < 9; ++q) R.H[0][0][q] = (q % 4 == 0) ? 2.0 : 0.0;
}

// s = |r|^2 - (r.e)^2 / |e|^2
__device__ inline void red_pe(Red& R, d3 r, d3 e) {
  R.nv = 2;
  double c = dot(r, e), q = dot(e, e), iq = 1.0 / q;
  R.g[0] = 2.0 * r - (2.0 * c * iq) * e;
  R.g[1] = (-2.0 * c * iq) * r + (2.0 * c * c * iq * iq) * e;
  double rv[3] = {r.x, r.y, r.z}, ev[3] = {e.x, e.y, e.z};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double dij = (i == j) ? 1.0 : 0.0;
      R.H[0][0][3 * i + j] = 2.0 * dij - 2.0 * ev[i] * ev[j] * iq;
      R.H[0][1][3 * i + j] = -2.0 * (ev[i] * rv[j] + c * dij) * iq + 4.0 * c * ev[i] * ev[j] * iq * iq;
      R.H[1][1][3 * i + j] = -2.0 * rv[i] * rv[j] * iq + 4.0 * c * (rv[i] * ev[j] + ev[i] * rv[j]) * iq * iq +
                             2.0 * c * c * dij * iq * iq - 8.0 * c * c * ev[i] * ev[j] * iq * iq * iq;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R.H[1][0][3 * i + j] = R.H[0][1][3 * j + i];
}

// s = (v.n)^2 / |n|^2, n = a x b
__device__ inline void red_plane(Red& R, d3 v, d3 a, d3 b) {
  R.nv = 3;
  d3 n = cross(a, b);
  double c = dot(v, n), q = dot(n, n), iq = 1.0 / q;
  d3 gn = (2.0 * c * iq) * v - (2.0 * c * c * iq * iq) * n;
  R.g[0] = (2.0 * c * iq) * n;
  R.g[1] = cross(b, gn);
  R.g[2] = cross(gn, a);
  double vv[3] = {v.x, v.y, v.z}, nv[3] = {n.x, n.y, n.z};
  double Gvn[9], Gnn[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double dij = (i == j) ? 1.0 : 0.0;
      R.H[0][0][3 * i + j] = 2.0 * nv[i] * nv[j] * iq;
      Gvn[3 * i + j] = 2.0 * (nv[i] * vv[j] + c * dij) * iq - 4.0 * c * nv[i] * nv[j] * iq * iq;
      Gnn[3 * i + j] = 2.0 * vv[i] * vv[j] * iq - 4.0 * c * (vv[i] * nv[j] + nv[i] * vv[j]) * iq * iq -
                       2.0 * c * c * dij * iq * iq + 8.0 * c * c * nv[i] * nv[j] * iq * iq * iq;
    }
  double Sa[9], Sb[9], Sg[9], mSb[9], mSa[9], T[9], T2[9];
  skew9(a, Sa);
  skew9(b, Sb);
  skew9(gn, Sg);
  for (int i = 0; i < 9; ++i) { mSb[i] = -Sb[i]; mSa[i] = -Sa[i]; }
  mm3(Gvn, mSb, R.H[0][1]);
  mm3(Gvn, Sa, R.H[0][2]);
  mm3(Sb, Gnn, T);
  mm3(T, mSb, R.H[1][1]);
  mm3(T, Sa, T2);
  for (int i = 0; i < 9; ++i) R.H[1][2][i] = T2[i] - Sg[i];
  mm3(mSa, Gnn, T);
  mm3(T, Sa, R.H[2][2]);
  for (int m = 0; m < 3; ++m)
    for (int nn = 0; nn < m; ++nn)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R.H[m][nn][3 * i + j] = R.H[nn][m][3 * j + i];
}

__device__ inline void red_setC(Red& R, int m, int k0, double c0, int k1, double c1) {
  for (int k = 0; k < 4; ++k) R.C[m][k] = 0.0;
  R.C[m][k0] = c0;
  if (k1 >= 0) R.C[m][k1] += c1;
}

// Reduced derivatives of the squared distance of (kind, type).
__device__ inline void dist_reduced(int kind, int type, const d3* x, Red& R, double& s) {
  if (kind == 0) {
    if (type <= 2) {
      d3 d = x[0] - x[1 + type];
      s = dot(d, d);
      red_pp(R, d);
      red_setC(R, 0, 0, 1.0, 1 + type, -1.0);
    } else if (type <= 5) {
      int i0 = 1 + (type - 3), i1 = 1 + (type - 2) % 3;
      d3 r = x[0] - x[i0], e = x[i1] - x[i0];
      double c = dot(r, e);
      s = dot(r, r) - c * c / dot(e, e);
      red_pe(R, r, e);
      red_setC(R, 0, 0, 1.0, i0, -1.0);
      red_setC(R, 1, i1, 1.0, i0, -1.0);
    } else {
      d3 v = x[0] - x[1], a = x[2] - x[1], b = x[3] - x[1];
      d3 n = cross(a, b);
      double c = dot(v, n);
      s = c * c / dot(n, n);
      red_plane(R, v, a, b);
      red_setC(R, 0, 0, 1.0, 1, -1.0);
      red_setC(R, 1, 2, 1.0, 1, -1.0);
      red_setC(R, 2, 3, 1.0, 1, -1.0);
    }
  } else {
    if (type <= 3) {
      int ia = type / 2, ib = 2 + type % 2;
      d3 d = x[ia] - x[ib];
      s = dot(d, d);
      red_pp(R, d);
      red_setC(R, 0, ia, 1.0, ib, -1.0);
    } else if (type <= 7) {
      const int pt[4] = {2, 3, 0, 1}, e0[4] = {0, 0, 2, 2}, e1[4] = {1, 1, 3, 3};
      int c_ = type - 4;
      d3 r = x[pt[c_]] - x[e0[c_]], e = x[e1[c_]] - x[e0[c_]];
      double c = dot(r, e);
      s = dot(r, r) - c * c / dot(e, e);
      red_pe(R, r, e);
      red_setC(R, 0, pt[c_], 1.0, e0[c_], -1.0);
      red_setC(R, 1, e1[c_], 1.0, e0[c_], -1.0);
    } else {
      d3 v = x[0] - x[2], a = x[1] - x[0], b = x[3] - x[2];
      d3 n = cross(a, b);
      double c = dot(v, n);
      s = c * c / dot(n, n);
      red_plane(R, v, a, b);
      red_setC(R, 0, 0, 1.0, 2, -1.0);
      red_setC(R, 1, 1, 1.0, 0, -1.0);
      red_setC(R, 2, 3, 1.0, 2, -1.0);
    }
  }
}

// Expand reduced derivatives to the 12-DOF gradient and Hessian.
__device__ inline void red_expand(const Red& R, double* g, double* H) {
  for (int k = 0; k < 4; ++k) {
    d3 acc = mk(0, 0, 0);
    for (int m = 0; m < R.nv; ++m) acc = acc + R.C[m][k] * R.g[m];
    g[3 * k] = acc.x; g[3 * k + 1] = acc.y; g[3 * k + 2] = acc.z;
  }
  if (!H) return;
  for (int k = 0; k < 4; ++k)
    for (int l = 0; l < 4; ++l) {
      double blk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      for (int m = 0; m < R.nv; ++m) {
        double cmk = R.C[m][k];
        if (cmk == 0.0) continue;
        for (int n = 0; n < R.nv; ++n) {
          double c = cmk * R.C[n][l];
          if (c == 0.0) continue;
          for (int q = 0; q < 9; ++q) blk[q] += c * R.H[m][n][q];
        }
      }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[12 * (3 * k + i) + 3 * l + j] = blk[3 * i + j];
    }
}

}  // namespace ipc
