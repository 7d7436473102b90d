// Plain CPU restatement of the path tracer of the simulated frames (§III-D.2)
// with the shadow-receiving background material (§III-D.3, Eq. 7).
//
// TEST INFRASTRUCTURE ONLY: only the tests use it; it shares no code with the
// CUDA library.  Closest hits by brute force over every triangle (no
// acceleration structure); FP32 arithmetic compiled with -ffp-contract=off.
//
// The estimator (what a pixel's value is): the mean over `spp` paths of the
// radiance carried to the camera, where a path
//   * starts at the eye through the pixel, jittered inside it;
//   * at an emissive triangle adds its radiance if it is the first hit, then
//     ends; at a transparent triangle continues straight on, its throughput
//     multiplied by the triangle's transmittance;
//   * at a background triangle ends with C_tex [1 - lambda_s (1 - V)] (Eq. 7),
//     V the fraction of n_shadow light samples visible from the point;
//   * at a diffuse triangle adds one light sample (a light triangle chosen in
//     proportion to area, a uniform point on it: radiance x albedo / pi x
//     cos cos' / d^2 x total light area, if visible), then, unless it is the
//     last vertex, continues in a cosine-distributed direction (a uniform
//     point of the unit disk by rejection, lifted to the hemisphere) with its
//     throughput multiplied by the albedo.
// The random numbers are the splitmix64 finaliser (Steele, Lea and Flood 2014)
// of (seed, pixel, sample, dimension), 24 bits each, dimension 0 and 1 the
// pixel jitter, then 64 dimensions per path vertex.
#include <cmath>
#include <cstdint>
#include <vector>

namespace {

struct V3 { float x, y, z; };
inline V3 v3(float a, float b, float c) { return V3{a, b, c}; }
inline V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
inline V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
inline V3 operator*(float s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
inline V3 times(V3 a, V3 b) { return v3(a.x * b.x, a.y * b.y, a.z * b.z); }
inline float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
inline V3 unit(V3 a) { return (1.0f / std::sqrt(dot(a, a))) * a; }

uint64_t splitmix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
float rnd(uint64_t key, unsigned dim) { return (float)(splitmix(key + dim) >> 40) * (1.0f / 16777216.0f); }

enum { DIFFUSE = 0, EMISSIVE = 1, BACKGROUND = 2, TRANSPARENT = 3 };

struct Frame {
  int nt;
  const int* tri;
  const int* type;
  const float* rgb;
  std::vector<V3> x;
  std::vector<int> lights;
  std::vector<float> cum;  // cumulative light areas
};

V3 vert(const Frame& F, int t, int k) { return F.x[F.tri[3 * t + k]]; }

// Moller-Trumbore in the order of its definition
bool meet(V3 o, V3 d, V3 a, V3 b, V3 c, float& t) {
  V3 e1 = b - a, e2 = c - a;
  V3 p = cross(d, e2);
  float det = dot(e1, p);
  if (det == 0.0f) return false;
  float inv = 1.0f / det;
  V3 tv = o - a;
  float u = dot(tv, p) * inv;
  if (u < 0.0f || u > 1.0f) return false;
  V3 q = cross(tv, e1);
  float v = dot(d, q) * inv;
  if (v < 0.0f || u + v > 1.0f) return false;
  t = dot(e2, q) * inv;
  return true;
}

// closest triangle with t > eps; on equal t the first in index order
int first_hit(const Frame& F, V3 o, V3 d, float eps, float& tbest) {
  int best = -1;
  tbest = INFINITY;
  for (int t = 0; t < F.nt; ++t) {
    float tt;
    if (meet(o, d, vert(F, t, 0), vert(F, t, 1), vert(F, t, 2), tt) && tt > eps && tt < tbest) {
      tbest = tt;
      best = t;
    }
  }
  return best;
}

bool unblocked(const Frame& F, V3 o, V3 y) {
  V3 d = y - o;
  for (int t = 0; t < F.nt; ++t) {
    if (F.type[t] == EMISSIVE || F.type[t] == TRANSPARENT) continue;
    float tt;
    if (meet(o, d, vert(F, t, 0), vert(F, t, 1), vert(F, t, 2), tt) && tt > 0.0f && tt < 1.0f) return false;
  }
  return true;
}

int light_point(const Frame& F, float u0, float u1, float u2, V3& y, V3& ny) {
  const int n = (int)F.lights.size();
  float target = u0 * F.cum[n];
  int k = 0;
  while (k < n - 1 && !(F.cum[k + 1] > target)) ++k;
  int t = F.lights[k];
  V3 a = vert(F, t, 0), b = vert(F, t, 1), c = vert(F, t, 2);
  float s = std::sqrt(u1);
  float b0 = 1.0f - s, b1 = u2 * s;
  y = (b0 * a + b1 * b) + (1.0f - b0 - b1) * c;
  ny = unit(cross(b - a, c - a));
  return t;
}

}  // namespace

extern "C" {

// image (height, width, 3) of the frame; cam = eye[3], fwd[3], right[3], up[3], tan_half_fov
void orc_render(int nv, const double* x, int nt, const int* tri, const int* type, const float* rgb, const float* cam,
                int width, int height, int spp, int max_depth, int n_shadow, float lambda_s, float eps,
                unsigned long long seed, float* img) {
  Frame F;
  F.nt = nt;
  F.tri = tri;
  F.type = type;
  F.rgb = rgb;
  F.x.resize(nv);
  for (int i = 0; i < nv; ++i) F.x[i] = v3((float)x[3 * i], (float)x[3 * i + 1], (float)x[3 * i + 2]);
  F.cum.push_back(0.0f);
  for (int t = 0; t < nt; ++t)
    if (type[t] == EMISSIVE) {
      F.lights.push_back(t);
      V3 cr = cross(vert(F, t, 1) - vert(F, t, 0), vert(F, t, 2) - vert(F, t, 0));
      F.cum.push_back(F.cum.back() + 0.5f * std::sqrt(dot(cr, cr)));
    }
  const int nl = (int)F.lights.size();
  const V3 eye = v3(cam[0], cam[1], cam[2]), fwd = v3(cam[3], cam[4], cam[5]), rgt = v3(cam[6], cam[7], cam[8]),
           upv = v3(cam[9], cam[10], cam[11]);
  const float tf = cam[12];
  const float aspect = (float)width / (float)height;
  for (int py = 0; py < height; ++py)
    for (int px = 0; px < width; ++px) {
      const int pix = py * width + px;
      const uint64_t kp = splitmix(seed ^ splitmix((uint64_t)pix));
      V3 sum = v3(0.0f, 0.0f, 0.0f);
      for (int s = 0; s < spp; ++s) {
        const uint64_t key = splitmix(kp ^ (uint64_t)s);
        float sx = (((float)px + rnd(key, 0)) / (float)width * 2.0f - 1.0f) * tf * aspect;
        float sy = (1.0f - ((float)py + rnd(key, 1)) / (float)height * 2.0f) * tf;
        V3 o = eye;
        V3 d = unit((fwd + sx * rgt) + sy * upv);
        V3 thr = v3(1.0f, 1.0f, 1.0f), L = v3(0.0f, 0.0f, 0.0f);
        for (int depth = 0; depth <= max_depth; ++depth) {
          const unsigned base = 2 + (unsigned)depth * 64;
          float t;
          const int h = first_hit(F, o, d, eps, t);
          if (h < 0) break;
          const V3 col = v3(rgb[3 * h], rgb[3 * h + 1], rgb[3 * h + 2]);
          const V3 p = o + t * d;
          if (type[h] == EMISSIVE) {
            if (depth == 0) L = L + times(thr, col);
            break;
          }
          if (type[h] == TRANSPARENT) {
            thr = times(thr, col);
            o = p;
            continue;
          }
          V3 n = unit(cross(vert(F, h, 1) - vert(F, h, 0), vert(F, h, 2) - vert(F, h, 0)));
          if (dot(n, d) > 0.0f) n = -1.0f * n;
          const V3 po = p + eps * n;
          if (type[h] == BACKGROUND) {
            int seen = 0;
            if (nl > 0)
              for (int k = 0; k < n_shadow; ++k) {
                V3 y, ny;
                light_point(F, rnd(key, base + 3 * k), rnd(key, base + 3 * k + 1), rnd(key, base + 3 * k + 2), y, ny);
                if (unblocked(F, po, y)) ++seen;
              }
            const float V = n_shadow > 0 ? (float)seen / (float)n_shadow : 1.0f;
            L = L + times(thr, (1.0f - lambda_s * (1.0f - V)) * col);
            break;
          }
          if (nl > 0) {
            V3 y, ny;
            const int lt = light_point(F, rnd(key, base), rnd(key, base + 1), rnd(key, base + 2), y, ny);
            const V3 w = y - po;
            const float d2 = dot(w, w);
            const V3 wn = (1.0f / std::sqrt(d2)) * w;
            const float cp = dot(n, wn);
            float cl = -dot(ny, wn);
            if (cl < 0.0f) cl = -cl;
            if (cp > 0.0f && unblocked(F, po, y)) {
              const float g = cp * cl / d2 * F.cum[nl] * (1.0f / 3.14159265f);
              const V3 le = v3(rgb[3 * lt], rgb[3 * lt + 1], rgb[3 * lt + 2]);
              L = L + times(thr, g * times(col, le));
            }
          }
          if (depth == max_depth) break;
          float dx = 0.0f, dy = 0.0f;
          for (int k = 0; k < 16; ++k) {
            const float a = 2.0f * rnd(key, base + 3 + 2 * k) - 1.0f, b = 2.0f * rnd(key, base + 4 + 2 * k) - 1.0f;
            if (a * a + b * b < 1.0f) { dx = a; dy = b; break; }
          }
          const float dz = std::sqrt(std::fmax(0.0f, 1.0f - dx * dx - dy * dy));
          const V3 hv = (n.x > 0.9f || n.x < -0.9f) ? v3(0.0f, 1.0f, 0.0f) : v3(1.0f, 0.0f, 0.0f);
          const V3 t1 = unit(cross(hv, n));
          const V3 t2 = cross(n, t1);
          d = unit((dx * t1 + dy * t2) + dz * n);
          o = po;
          thr = times(thr, col);
        }
        sum = sum + L;
      }
      const float inv = 1.0f / (float)spp;
      img[3 * pix] = sum.x * inv;
      img[3 * pix + 1] = sum.y * inv;
      img[3 * pix + 2] = sum.z * inv;
    }
}

}  // extern "C"
