// Physics-to-render dual-mesh mapping (§III-D.1, Eqs. 5-6).
//
// The render mesh of a deformable body is its simulation surface after L
// levels of Loop subdivision.  Every level is linear in the vertex positions,
// so the L levels compose into one sparse matrix W (N_fine x N_coarse, Eq. 5)
// built once on the host, and each frame's fine positions are one sparse
// product X_f = W X_c (Eq. 6) on the device.
//
// Loop's rules per level: an edge (a, b) with opposite vertices c, d gets the
// new vertex 3/8 (a + b) + 1/8 (c + d) (a boundary edge: the midpoint); an old
// vertex of valence n moves to (1 - n beta) v + beta * (sum of neighbours),
// beta = (5/8 - (3/8 + cos(2 pi / n) / 4)^2) / n (a boundary vertex:
// 3/4 v + 1/8 of each boundary neighbour); each triangle splits into four.
// New vertices follow the old ones, one per edge in increasing (min, max)
// vertex order.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>
#include "../../include/ipcsim.h"
#include "kernels.h"

struct ipc_dual_mesh {
  int n_coarse = 0, n_fine = 0, levels = 0;
  long long nnz = 0;
  std::vector<int> fine_tris;
  std::vector<int> h_row, h_col;
  std::vector<double> h_val;
  int* row = nullptr;
  int* col = nullptr;
  double* val = nullptr;
};

namespace {

thread_local std::string g_dual_error;

// sparse rows: (column, weight), columns sorted and unique
using Row = std::vector<std::pair<int, double>>;

struct Level {
  std::vector<Row> rows;    // weights of the new vertices on the old ones
  std::vector<int> tris;    // the new triangles
  int n_new = 0;
};

Level subdivide_once(const std::vector<int>& tris, int n) {
  const int nt = (int)tris.size() / 3;
  // every triangle side as (min, max, opposite vertex), sorted by the edge
  struct Side { int a, b, opp; };
  std::vector<Side> sides;
  sides.reserve(3 * (size_t)nt);
  for (int t = 0; t < nt; ++t)
    for (int k = 0; k < 3; ++k) {
      const int u = tris[3 * t + k], v = tris[3 * t + (k + 1) % 3], w = tris[3 * t + (k + 2) % 3];
      sides.push_back({std::min(u, v), std::max(u, v), w});
    }
  std::sort(sides.begin(), sides.end(), [](const Side& x, const Side& y) {
    return x.a != y.a ? x.a < y.a : (x.b != y.b ? x.b < y.b : x.opp < y.opp);
  });
  // unique edges with up to two opposite vertices
  struct Edge { int a, b, o0, o1; };
  std::vector<Edge> edges;
  for (size_t i = 0; i < sides.size();) {
    size_t j = i;
    while (j < sides.size() && sides[j].a == sides[i].a && sides[j].b == sides[i].b) ++j;
    Edge e{sides[i].a, sides[i].b, sides[i].opp, j - i >= 2 ? sides[i + 1].opp : -1};
    edges.push_back(e);
    i = j;
  }
  Level L;
  L.n_new = n + (int)edges.size();
  L.rows.assign(L.n_new, Row());
  // neighbourhoods of the old vertices
  std::vector<std::vector<int>> nb(n), bnb(n);
  for (const Edge& e : edges) {
    nb[e.a].push_back(e.b);
    nb[e.b].push_back(e.a);
    if (e.o1 < 0) {
      bnb[e.a].push_back(e.b);
      bnb[e.b].push_back(e.a);
    }
  }
  for (int v = 0; v < n; ++v) {
    Row& r = L.rows[v];
    if (bnb[v].size() >= 2) {
      r.push_back({v, 0.75});
      r.push_back({bnb[v][0], 0.125});
      r.push_back({bnb[v][1], 0.125});
    } else if (!nb[v].empty()) {
      const int val = (int)nb[v].size();
      const double c = 0.375 + 0.25 * std::cos(2.0 * M_PI / val);
      const double beta = (0.625 - c * c) / val;
      r.push_back({v, 1.0 - val * beta});
      for (int u : nb[v]) r.push_back({u, beta});
    } else {
      r.push_back({v, 1.0});
    }
    std::sort(r.begin(), r.end());
  }
  for (size_t k = 0; k < edges.size(); ++k) {
    const Edge& e = edges[k];
    Row& r = L.rows[n + k];
    if (e.o1 >= 0) {
      r = {{e.a, 0.375}, {e.b, 0.375}, {e.o0, 0.125}, {e.o1, 0.125}};
    } else {
      r = {{e.a, 0.5}, {e.b, 0.5}};
    }
    std::sort(r.begin(), r.end());
    // a vertex that is also an opposite vertex (degenerate meshes): merge duplicates
    Row m;
    for (auto& p : r) {
      if (!m.empty() && m.back().first == p.first) m.back().second += p.second;
      else m.push_back(p);
    }
    r.swap(m);
  }
  auto edge_vertex = [&](int u, int v) {
    const int a = std::min(u, v), b = std::max(u, v);
    const auto it = std::lower_bound(edges.begin(), edges.end(), Edge{a, b, 0, 0},
                                     [](const Edge& x, const Edge& y) { return x.a != y.a ? x.a < y.a : x.b < y.b; });
    return n + (int)(it - edges.begin());
  };
  L.tris.reserve(12 * (size_t)nt);
  for (int t = 0; t < nt; ++t) {
    const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
    const int ab = edge_vertex(a, b), bc = edge_vertex(b, c), ca = edge_vertex(c, a);
    const int quad[12] = {a, ab, ca, b, bc, ab, c, ca, bc, ab, bc, ca};
    L.tris.insert(L.tris.end(), quad, quad + 12);
  }
  return L;
}

// rows of S W (Gustavson: one dense accumulator, the touched columns sorted per row)
std::vector<Row> compose(const std::vector<Row>& S, const std::vector<Row>& W, int n_cols) {
  std::vector<Row> out(S.size());
  std::vector<double> acc(n_cols, 0.0);
  std::vector<char> used(n_cols, 0);
  std::vector<int> touched;
  for (size_t i = 0; i < S.size(); ++i) {
    touched.clear();
    for (const auto& sk : S[i])
      for (const auto& wk : W[sk.first]) {
        if (!used[wk.first]) { used[wk.first] = 1; touched.push_back(wk.first); }
        acc[wk.first] += sk.second * wk.second;
      }
    std::sort(touched.begin(), touched.end());
    Row& r = out[i];
    r.reserve(touched.size());
    for (int c : touched) {
      r.push_back({c, acc[c]});
      acc[c] = 0.0;
      used[c] = 0;
    }
  }
  return out;
}

// X_f = W X_c: a group of 4 lanes per fine vertex, lanes over the row's entries, shuffle sum
__global__ void k_dual_apply(int n_fine, const int* __restrict__ row, const int* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ xc, double* __restrict__ xf) {
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 2, lane = threadIdx.x & 3;
  const bool live = g < n_fine;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (live) {
    for (int k = row[g] + lane; k < row[g + 1]; k += 4) {
      const int c = col[k];
      const double w = val[k];
      s0 = fma(w, xc[3 * c], s0);
      s1 = fma(w, xc[3 * c + 1], s1);
      s2 = fma(w, xc[3 * c + 2], s2);
    }
  }
  for (int o = 2; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o, 4);
    s1 += __shfl_down_sync(0xffffffffu, s1, o, 4);
    s2 += __shfl_down_sync(0xffffffffu, s2, o, 4);
  }
  if (live && lane == 0) {
    xf[3 * (size_t)g] = s0;
    xf[3 * (size_t)g + 1] = s1;
    xf[3 * (size_t)g + 2] = s2;
  }
}

}  // namespace

extern "C" {

ipc_status sim_dual_mesh_create(const int* tris_host, int n_tris, int n_verts, int levels, int upload,
                                ipc_dual_mesh** out) {
  if (!out) return IPC_ERR_ARG;
  *out = nullptr;
  if (!tris_host || n_tris <= 0 || n_verts <= 0 || levels < 0 || levels > 6) {
    g_dual_error = "sim_dual_mesh_create: need triangles, vertices and 0 <= levels <= 6";
    return IPC_ERR_ARG;
  }
  std::vector<int> tris(tris_host, tris_host + 3 * (size_t)n_tris);
  for (int v : tris)
    if (v < 0 || v >= n_verts) { g_dual_error = "sim_dual_mesh_create: vertex id out of range"; return IPC_ERR_ARG; }
  std::vector<Row> W(n_verts);
  for (int v = 0; v < n_verts; ++v) W[v] = {{v, 1.0}};
  int n = n_verts;
  for (int l = 0; l < levels; ++l) {
    Level L = subdivide_once(tris, n);
    W = compose(L.rows, W, n_verts);
    tris.swap(L.tris);
    n = L.n_new;
  }
  ipc_dual_mesh* m = new ipc_dual_mesh();
  m->n_coarse = n_verts;
  m->n_fine = n;
  m->levels = levels;
  m->fine_tris = tris;
  m->h_row.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) m->h_row[i + 1] = m->h_row[i] + (int)W[i].size();
  m->nnz = m->h_row[n];
  m->h_col.reserve(m->nnz);
  m->h_val.reserve(m->nnz);
  for (const Row& r : W)
    for (const auto& p : r) { m->h_col.push_back(p.first); m->h_val.push_back(p.second); }
  if (!upload) {
    *out = m;
    return IPC_OK;
  }
  cudaError_t e = cudaMalloc(&m->row, sizeof(int) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&m->col, sizeof(int) * std::max<long long>(m->nnz, 1));
  if (e == cudaSuccess) e = cudaMalloc(&m->val, sizeof(double) * std::max<long long>(m->nnz, 1));
  if (e == cudaSuccess) e = cudaMemcpy(m->row, m->h_row.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->col, m->h_col.data(), sizeof(int) * m->nnz, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->val, m->h_val.data(), sizeof(double) * m->nnz, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    g_dual_error = std::string("sim_dual_mesh_create: ") + cudaGetErrorString(e);
    sim_dual_mesh_destroy(m);
    return IPC_ERR_CUDA;
  }
  *out = m;
  return IPC_OK;
}

ipc_status sim_dual_mesh_sizes(const ipc_dual_mesh* m, long long* out4) {
  if (!m || !out4) return IPC_ERR_ARG;
  out4[0] = m->n_coarse;
  out4[1] = m->n_fine;
  out4[2] = (long long)m->fine_tris.size() / 3;
  out4[3] = m->nnz;
  return IPC_OK;
}

ipc_status sim_dual_mesh_topology(const ipc_dual_mesh* m, int* fine_tris_host, int* row_host, int* col_host,
                                  double* val_host) {
  if (!m) return IPC_ERR_ARG;
  if (fine_tris_host) std::copy(m->fine_tris.begin(), m->fine_tris.end(), fine_tris_host);
  if (row_host) std::copy(m->h_row.begin(), m->h_row.end(), row_host);
  if (col_host) std::copy(m->h_col.begin(), m->h_col.end(), col_host);
  if (val_host) std::copy(m->h_val.begin(), m->h_val.end(), val_host);
  return IPC_OK;
}

ipc_status sim_dual_mesh_apply(const ipc_dual_mesh* m, const double* xc_dev, double* xf_dev, void* stream) {
  if (!m || !xc_dev || !xf_dev || !m->row) return IPC_ERR_ARG;
  const int threads = 256;
  const long long lanes = 4LL * m->n_fine;
  k_dual_apply<<<(unsigned)((lanes + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(
      m->n_fine, m->row, m->col, m->val, xc_dev, xf_dev);
  ipc::count_launch();
  return cudaGetLastError() == cudaSuccess ? IPC_OK : IPC_ERR_CUDA;
}

const char* sim_dual_mesh_last_error(void) { return g_dual_error.c_str(); }

void sim_dual_mesh_destroy(ipc_dual_mesh* m) {
  if (!m) return;
  cudaFree(m->row);
  cudaFree(m->col);
  cudaFree(m->val);
  delete m;
}

}  // extern "C"
