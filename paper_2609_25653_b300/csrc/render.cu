// Headless CUDA path tracer with the appearance-preserving shadow-receiving
// background material (§III-D.2 and §III-D.3, Eq. 7).
//
// Every frame renders the simulated surfaces at their current positions:
// the triangles are put into an LBVH (the same construction as the contact
// broad phase, FP32 node boxes rounded outward), and one thread per pixel
// traces `spp` paths of at most `max_depth` diffuse bounces with next-event
// estimation toward the area lights (emissive triangles, sampled in
// proportion to their area).  A path that reaches a background triangle
// ends there with the colour of Eq. 7,
//     C_bg = C_tex [1 - lambda_s (1 - V)],
// where V is the fraction of `n_shadow` light samples visible from the hit
// point: the reconstructed texture is kept as it is (no BRDF, no second
// illumination) and only the shadows of the simulated objects darken it.
// Transparent triangles are thin sheets: a path passes through them with its
// throughput multiplied by their transmittance (they cast no shadows).
//
// Every random number is a counter-based hash (the splitmix64 finaliser of
// Steele, Lea and Flood) of the seed, the pixel, the sample and the sampling
// dimension, so a frame is a deterministic function of its inputs; the
// arithmetic is FP32, compiled without contraction (-fmad=false), so that a
// CPU restatement with the same operation order reproduces it.  The output is
// linear RGB (no tone mapping).
#include <cuda_runtime.h>
#include <algorithm>
#include <string>
#include <vector>
#include "../../include/ipcsim.h"
#include "bvh.cuh"
#include "kernels.h"

struct ipc_render {
  int nv = 0, nt = 0, n_lights = 0;
  int* tris = nullptr;       // (nt, 3)
  int* type = nullptr;       // (nt)
  float* rgb = nullptr;      // (nt, 3)
  int* lights = nullptr;     // (n_lights) emissive triangles
  float* cdf = nullptr;      // (n_lights + 1) cumulative light areas (last: total)
  float* xf = nullptr;       // (nv, 3) FP32 positions of the frame
  ipc::Bvh tree;
  ipc::DevAlloc mem;
};

namespace {

thread_local std::string g_render_error;

struct f3 { float x, y, z; };
__device__ inline f3 mkf(float a, float b, float c) { return f3{a, b, c}; }
__device__ inline f3 add(f3 a, f3 b) { return mkf(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ inline f3 sub(f3 a, f3 b) { return mkf(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ inline f3 mul(float s, f3 a) { return mkf(s * a.x, s * a.y, s * a.z); }
__device__ inline f3 hadamard(f3 a, f3 b) { return mkf(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ inline float dotf(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline f3 crossf(f3 a, f3 b) { return mkf(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
__device__ inline f3 normalizef(f3 a) { return mul(1.0f / sqrtf(dotf(a, a)), a); }
__device__ inline f3 ldf(const float* p, int i) { return mkf(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }

// splitmix64 finaliser (Steele, Lea and Flood, OOPSLA 2014)
__device__ inline unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// uniform in [0, 1) with 24 random bits
__device__ inline float uniform(unsigned long long key, unsigned dim) {
  return (float)(mix64(key + dim) >> 40) * (1.0f / 16777216.0f);
}

struct Hit { float t; int tri; };

// Moller-Trumbore; true with the ray parameter t when the ray o + t d meets triangle (a, b, c)
__device__ inline bool ray_tri(f3 o, f3 d, f3 a, f3 b, f3 c, float& t) {
  const f3 e1 = sub(b, a), e2 = sub(c, a);
  const f3 p = crossf(d, e2);
  const float det = dotf(e1, p);
  if (det == 0.0f) return false;
  const float inv = 1.0f / det;
  const f3 tv = sub(o, a);
  const float u = dotf(tv, p) * inv;
  if (u < 0.0f || u > 1.0f) return false;
  const f3 q = crossf(tv, e1);
  const float v = dotf(d, q) * inv;
  if (v < 0.0f || u + v > 1.0f) return false;
  t = dotf(e2, q) * inv;
  return true;
}

// conservative slab test of a node box (the far end is widened by a few ulps)
__device__ inline bool ray_box(f3 o, f3 inv, const float* b, float tmax) {
  float t0 = 0.0f, t1 = tmax;
  const float ov[3] = {o.x, o.y, o.z}, iv[3] = {inv.x, inv.y, inv.z};
  for (int k = 0; k < 3; ++k) {
    float ta = (b[k] - ov[k]) * iv[k], tb = (b[3 + k] - ov[k]) * iv[k];
    if (ta > tb) { const float s = ta; ta = tb; tb = s; }
    tb *= 1.0000004f;
    if (ta != ta) ta = -INFINITY;  // 0 * inf: the ray runs inside this slab's plane
    if (tb != tb) tb = INFINITY;
    t0 = ta > t0 ? ta : t0;
    t1 = tb < t1 ? tb : t1;
    if (t0 > t1) return false;
  }
  return true;
}

struct Scene {
  int n;
  const int* prim;
  const int* left;
  const int* right;
  const float* box;
  const int* tris;
  const int* type;
  const float* rgb;
  const float* x;
  const int* lights;
  const float* cdf;
  int n_lights;
};

// closest hit with t > eps (ties: the smaller triangle index); kinds listed in `skip_transparent` pass
__device__ inline Hit closest(const Scene& S, f3 o, f3 d, float eps) {
  Hit h{INFINITY, -1};
  if (S.n <= 0) return h;
  const f3 inv = mkf(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  int stack[64];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const int node = stack[--sp];
    if (!ray_box(o, inv, S.box + 6 * (size_t)node, h.t)) continue;
    if (node >= S.n - 1) {
      const int t = S.prim[node - (S.n - 1)];
      const int* v = S.tris + 3 * t;
      float tt;
      if (ray_tri(o, d, ldf(S.x, v[0]), ldf(S.x, v[1]), ldf(S.x, v[2]), tt) && tt > eps &&
          (tt < h.t || (tt == h.t && t < h.tri))) {
        h.t = tt;
        h.tri = t;
      }
    } else if (sp + 2 <= 64) {
      stack[sp++] = S.right[node];
      stack[sp++] = S.left[node];
    }
  }
  return h;
}

// true when no opaque triangle (diffuse or background) meets the segment o + t (y - o), 0 < t < 1 (the
// origin is already offset from its surface; lights and transparent sheets do not block)
__device__ inline bool visible(const Scene& S, f3 o, f3 y) {
  const f3 d = sub(y, o);
  const f3 inv = mkf(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  int stack[64];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const int node = stack[--sp];
    if (!ray_box(o, inv, S.box + 6 * (size_t)node, 1.0f)) continue;
    if (node >= S.n - 1) {
      const int t = S.prim[node - (S.n - 1)];
      const int ty = S.type[t];
      if (ty == IPC_MAT_EMISSIVE || ty == IPC_MAT_TRANSPARENT) continue;
      const int* v = S.tris + 3 * t;
      float tt;
      if (ray_tri(o, d, ldf(S.x, v[0]), ldf(S.x, v[1]), ldf(S.x, v[2]), tt) && tt > 0.0f && tt < 1.0f)
        return false;
    } else if (sp + 2 <= 64) {
      stack[sp++] = S.right[node];
      stack[sp++] = S.left[node];
    }
  }
  return true;
}

// a point on the lights, chosen in proportion to area; returns the light triangle
__device__ inline int sample_light(const Scene& S, float u0, float u1, float u2, f3& y, f3& ny) {
  const float total = S.cdf[S.n_lights];
  const float target = u0 * total;
  int lo = 0, hi = S.n_lights - 1;
  while (lo < hi) {  // first light whose cumulative area exceeds the target
    const int mid = (lo + hi) >> 1;
    if (S.cdf[mid + 1] > target) hi = mid; else lo = mid + 1;
  }
  const int t = S.lights[lo];
  const int* v = S.tris + 3 * t;
  const f3 a = ldf(S.x, v[0]), b = ldf(S.x, v[1]), c = ldf(S.x, v[2]);
  const float s = sqrtf(u1);
  const float b0 = 1.0f - s, b1 = u2 * s;
  y = add(add(mul(b0, a), mul(b1, b)), mul(1.0f - b0 - b1, c));
  ny = normalizef(crossf(sub(b, a), sub(c, a)));
  return t;
}

__device__ inline f3 tri_normal(const Scene& S, int t) {
  const int* v = S.tris + 3 * t;
  const f3 a = ldf(S.x, v[0]), b = ldf(S.x, v[1]), c = ldf(S.x, v[2]);
  return normalizef(crossf(sub(b, a), sub(c, a)));
}

// dimensions of the sampling sequence of one path vertex
constexpr unsigned DIMS_PER_BOUNCE = 64;

__global__ void k_render(Scene S, ipc_camera cam, ipc_render_params P, float* __restrict__ out) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_pix = cam.width * cam.height;
  if (px >= n_pix) return;
  const int ix = px % cam.width, iy = px / cam.width;
  const f3 eye = mkf(cam.eye[0], cam.eye[1], cam.eye[2]);
  const f3 fwd = mkf(cam.fwd[0], cam.fwd[1], cam.fwd[2]);
  const f3 rgt = mkf(cam.right[0], cam.right[1], cam.right[2]);
  const f3 upv = mkf(cam.up[0], cam.up[1], cam.up[2]);
  const float aspect = (float)cam.width / (float)cam.height;
  f3 acc = mkf(0.0f, 0.0f, 0.0f);
  const unsigned long long kp = mix64(P.seed ^ mix64((unsigned long long)px));
  for (int s = 0; s < P.spp; ++s) {
    const unsigned long long key = mix64(kp ^ (unsigned long long)s);
    const float jx = uniform(key, 0), jy = uniform(key, 1);
    const float sx = (((float)ix + jx) / (float)cam.width * 2.0f - 1.0f) * cam.tan_half_fov * aspect;
    const float sy = (1.0f - ((float)iy + jy) / (float)cam.height * 2.0f) * cam.tan_half_fov;
    f3 o = eye;
    f3 d = normalizef(add(add(fwd, mul(sx, rgt)), mul(sy, upv)));
    f3 thr = mkf(1.0f, 1.0f, 1.0f), L = mkf(0.0f, 0.0f, 0.0f);
    for (int depth = 0; depth <= P.max_depth; ++depth) {
      const unsigned base = 2 + (unsigned)depth * DIMS_PER_BOUNCE;
      const Hit h = closest(S, o, d, P.eps);
      if (h.tri < 0) break;
      const int ty = S.type[h.tri];
      const f3 col = ldf(S.rgb, h.tri);
      const f3 p = add(o, mul(h.t, d));
      if (ty == IPC_MAT_EMISSIVE) {
        if (depth == 0) L = add(L, hadamard(thr, col));  // later bounces count lights by next-event estimation
        break;
      }
      if (ty == IPC_MAT_TRANSPARENT) {
        thr = hadamard(thr, col);
        o = p;
        continue;
      }
      f3 n = tri_normal(S, h.tri);
      if (dotf(n, d) > 0.0f) n = mul(-1.0f, n);
      const f3 po = add(p, mul(P.eps, n));
      if (ty == IPC_MAT_BACKGROUND) {
        // Eq. 7: C_bg = C_tex [1 - lambda_s (1 - V)], V the visible fraction of n_shadow light samples
        int vis = 0;
        if (S.n_lights > 0)
          for (int k = 0; k < P.n_shadow; ++k) {
            f3 y, ny;
            sample_light(S, uniform(key, base + 3 * k), uniform(key, base + 3 * k + 1), uniform(key, base + 3 * k + 2),
                         y, ny);
            if (visible(S, po, y)) ++vis;
          }
        const float V = P.n_shadow > 0 ? (float)vis / (float)P.n_shadow : 1.0f;
        L = add(L, hadamard(thr, mul(1.0f - P.lambda_s * (1.0f - V), col)));
        break;
      }
      // diffuse: next-event estimation toward one light sample
      if (S.n_lights > 0) {
        f3 y, ny;
        const int lt = sample_light(S, uniform(key, base), uniform(key, base + 1), uniform(key, base + 2), y, ny);
        const f3 w = sub(y, po);
        const float d2 = dotf(w, w);
        const f3 wn = mul(1.0f / sqrtf(d2), w);
        const float cp = dotf(n, wn), cl = -dotf(ny, wn);
        const float clabs = cl < 0.0f ? -cl : cl;  // two-sided emitters
        if (cp > 0.0f && visible(S, po, y)) {
          const float g = cp * clabs / d2 * S.cdf[S.n_lights] * (1.0f / 3.14159265f);
          L = add(L, hadamard(thr, mul(g, hadamard(col, ldf(S.rgb, lt)))));
        }
      }
      if (depth == P.max_depth) break;
      // cosine-weighted bounce: a uniform point of the unit disk (rejection), lifted to the hemisphere
      float dx = 0.0f, dy = 0.0f;
      for (int k = 0; k < 16; ++k) {
        const float a = 2.0f * uniform(key, base + 3 + 2 * k) - 1.0f, b = 2.0f * uniform(key, base + 4 + 2 * k) - 1.0f;
        if (a * a + b * b < 1.0f) { dx = a; dy = b; break; }
      }
      const float dz = sqrtf(fmaxf(0.0f, 1.0f - dx * dx - dy * dy));
      const f3 hv = (n.x > 0.9f || n.x < -0.9f) ? mkf(0.0f, 1.0f, 0.0f) : mkf(1.0f, 0.0f, 0.0f);
      const f3 t1 = normalizef(crossf(hv, n));
      const f3 t2 = crossf(n, t1);
      d = normalizef(add(add(mul(dx, t1), mul(dy, t2)), mul(dz, n)));
      o = po;
      thr = hadamard(thr, col);
    }
    acc = add(acc, L);
  }
  const float inv = 1.0f / (float)P.spp;
  out[3 * (size_t)px] = acc.x * inv;
  out[3 * (size_t)px + 1] = acc.y * inv;
  out[3 * (size_t)px + 2] = acc.z * inv;
}

__global__ void k_to_f32(int n, const double* __restrict__ x, float* __restrict__ xf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * n) xf[i] = (float)x[i];
}

// cumulative areas of the light triangles, in order (one thread: the same sums as a serial loop)
__global__ void k_light_cdf(int n_lights, const int* __restrict__ lights, const int* __restrict__ tris,
                            const float* __restrict__ x, float* __restrict__ cdf) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  float c = 0.0f;
  cdf[0] = 0.0f;
  for (int k = 0; k < n_lights; ++k) {
    const int* v = tris + 3 * lights[k];
    const f3 a = ldf(x, v[0]), b = ldf(x, v[1]), cc = ldf(x, v[2]);
    const f3 cr = crossf(sub(b, a), sub(cc, a));
    c = c + 0.5f * sqrtf(dotf(cr, cr));
    cdf[k + 1] = c;
  }
}

}  // namespace

extern "C" {

ipc_status sim_render_create(const ipc_render_scene* d, ipc_render** out) {
  if (!out) return IPC_ERR_ARG;
  *out = nullptr;
  if (!d || d->n_verts <= 0 || d->n_tris <= 0 || !d->tris_host || !d->type_host || !d->rgb_host) {
    g_render_error = "sim_render_create: need vertices, triangles, types and colours";
    return IPC_ERR_ARG;
  }
  std::vector<int> lights;
  for (int t = 0; t < d->n_tris; ++t) {
    for (int k = 0; k < 3; ++k)
      if (d->tris_host[3 * t + k] < 0 || d->tris_host[3 * t + k] >= d->n_verts) {
        g_render_error = "sim_render_create: vertex id out of range";
        return IPC_ERR_ARG;
      }
    const int ty = d->type_host[t];
    if (ty < IPC_MAT_DIFFUSE || ty > IPC_MAT_TRANSPARENT) { g_render_error = "sim_render_create: unknown material"; return IPC_ERR_ARG; }
    if (ty == IPC_MAT_EMISSIVE) lights.push_back(t);
  }
  ipc_render* r = new ipc_render();
  r->nv = d->n_verts;
  r->nt = d->n_tris;
  r->n_lights = (int)lights.size();
  auto fail = [&](cudaError_t e) {
    g_render_error = std::string("sim_render_create: ") + cudaGetErrorString(e);
    sim_render_destroy(r);
    return IPC_ERR_CUDA;
  };
  cudaError_t e = cudaSuccess;
  auto get = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = r->mem.get(p, bytes); };
  get((void**)&r->tris, sizeof(int) * 3 * (size_t)r->nt);
  get((void**)&r->type, sizeof(int) * (size_t)r->nt);
  get((void**)&r->rgb, sizeof(float) * 3 * (size_t)r->nt);
  get((void**)&r->lights, sizeof(int) * std::max(1, r->n_lights));
  get((void**)&r->cdf, sizeof(float) * (r->n_lights + 1));
  get((void**)&r->xf, sizeof(float) * 3 * (size_t)r->nv);
  if (e != cudaSuccess) return fail(e);
  e = cudaMemcpy(r->tris, d->tris_host, sizeof(int) * 3 * (size_t)r->nt, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->type, d->type_host, sizeof(int) * (size_t)r->nt, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->rgb, d->rgb_host, sizeof(float) * 3 * (size_t)r->nt, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && r->n_lights)
    e = cudaMemcpy(r->lights, lights.data(), sizeof(int) * r->n_lights, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = ipc::bvh_alloc(r->tree, r->nt, r->mem);
  if (e != cudaSuccess) return fail(e);
  *out = r;
  return IPC_OK;
}

ipc_status sim_render_frame(ipc_render* r, const double* x_dev, const ipc_camera* cam, const ipc_render_params* p,
                            float* rgb_dev, void* stream) {
  if (!r || !x_dev || !cam || !p || !rgb_dev || cam->width <= 0 || cam->height <= 0 || p->spp <= 0 ||
      p->max_depth < 0 || p->n_shadow < 0)
    return IPC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // the tree over the frame's triangles (FP64 boxes of the positions, FP32 nodes rounded outward)
  ipc::bvh_leaf_boxes(st, r->tree, r->tris, 3, x_dev, nullptr, 0.0);
  ipc::bvh_build(st, r->tree);
  k_to_f32<<<(3 * r->nv + 255) / 256, 256, 0, st>>>(r->nv, x_dev, r->xf);
  k_light_cdf<<<1, 32, 0, st>>>(r->n_lights, r->lights, r->tris, r->xf, r->cdf);
  ipc::count_launch(2);
  Scene S{};
  S.n = r->tree.n;
  S.prim = r->tree.prim;
  S.left = r->tree.left;
  S.right = r->tree.right;
  S.box = r->tree.box;
  S.tris = r->tris;
  S.type = r->type;
  S.rgb = r->rgb;
  S.x = r->xf;
  S.lights = r->lights;
  S.cdf = r->cdf;
  S.n_lights = r->n_lights;
  const int n_pix = cam->width * cam->height;
  k_render<<<(n_pix + 127) / 128, 128, 0, st>>>(S, *cam, *p, rgb_dev);
  ipc::count_launch();
  return cudaGetLastError() == cudaSuccess ? IPC_OK : IPC_ERR_CUDA;
}

const char* sim_render_last_error(void) { return g_render_error.c_str(); }

void sim_render_destroy(ipc_render* r) {
  if (!r) return;
  cudaDeviceSynchronize();
  ipc::bvh_free(r->tree, r->mem);
  r->mem.put(r->tris, 0); r->mem.put(r->type, 0); r->mem.put(r->rgb, 0);
  r->mem.put(r->lights, 0); r->mem.put(r->cdf, 0); r->mem.put(r->xf, 0);
  delete r;
}

}  // extern "C"
