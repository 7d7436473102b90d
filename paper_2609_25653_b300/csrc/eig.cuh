// Symmetric PSD projection for small dense blocks (per tet 9x9, per pair up to 12x12).
//
// H <- V max(Lambda, 0) V^T by cyclic Jacobi rotations (Golub & Van Loan,
// "Matrix Computations", §8.5), run by one thread on a matrix in its local
// memory.  T = double on the FP64 path, float on the mixed path (Hessians
// only shape the Newton direction; gradients and energies stay FP64).
#pragma once
#include <cuda_runtime.h>

namespace ipc {

template <typename T>
__device__ inline T t_sqrt(T x);
template <>
__device__ inline double t_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ inline float t_sqrt<float>(float x) { return sqrtf(x); }

template <int N, typename T>
__device__ void jacobi_psd(T* A, T* V, T rel_tol) {
  for (int i = 0; i < N * N; ++i) V[i] = T(0);
  for (int i = 0; i < N; ++i) V[i * N + i] = T(1);
  T total = T(0);
  for (int i = 0; i < N * N; ++i) total += A[i] * A[i];
  if (total == T(0)) return;
  for (int sweep = 0; sweep < 30; ++sweep) {
    T off = T(0);
    for (int p = 0; p < N; ++p)
      for (int q = p + 1; q < N; ++q) off += T(2) * A[p * N + q] * A[p * N + q];
    if (off <= rel_tol * total) break;
    for (int p = 0; p < N - 1; ++p) {
      for (int q = p + 1; q < N; ++q) {
        T apq = A[p * N + q];
        if (apq == T(0)) continue;
        T theta = (A[q * N + q] - A[p * N + p]) / (T(2) * apq);
        T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + t_sqrt<T>(theta * theta + T(1)));
        T c = T(1) / t_sqrt<T>(t * t + T(1));
        T s = t * c;
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
          T akp = A[k * N + p], akq = A[k * N + q];
          A[k * N + p] = c * akp - s * akq;
          A[k * N + q] = s * akp + c * akq;
        }
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
          T apk = A[p * N + k], aqk = A[q * N + k];
          A[p * N + k] = c * apk - s * aqk;
          A[q * N + k] = s * apk + c * aqk;
        }
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
          T vkp = V[k * N + p], vkq = V[k * N + q];
          V[k * N + p] = c * vkp - s * vkq;
          V[k * N + q] = s * vkp + c * vkq;
        }
      }
    }
  }
}

// In-place PSD projection of the symmetric N x N matrix H (row-major).
// Skips the decomposition when every Gershgorin disc is non-negative.
template <int N, typename T>
__device__ void project_psd(T* H) {
  bool dominant = true;
  for (int i = 0; i < N && dominant; ++i) {
    T off = T(0);
    for (int j = 0; j < N; ++j)
      if (j != i) off += fabs(H[i * N + j]);
    if (H[i * N + i] < off) dominant = false;
  }
  if (dominant) return;
  T A[N * N], V[N * N];
  for (int i = 0; i < N * N; ++i) A[i] = H[i];
  jacobi_psd<N, T>(A, V, sizeof(T) == 8 ? T(1e-30) : T(1e-13));
  T lam[N];
  for (int k = 0; k < N; ++k) lam[k] = A[k * N + k] > T(0) ? A[k * N + k] : T(0);
  for (int i = 0; i < N; ++i)
    for (int j = i; j < N; ++j) {
      T s = T(0);
      for (int k = 0; k < N; ++k) s += V[i * N + k] * lam[k] * V[j * N + k];
      H[i * N + j] = s;
      H[j * N + i] = s;
    }
}


__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Parallel cyclic Jacobi PSD projection of the symmetric n x n matrix A (n
// even <= 12, row stride 12, shared memory) by one warp: n / 2 disjoint
// rotations per round (round-robin pairing), n - 1 rounds per sweep, then
// A <- V max(lambda, 0) V^T.  V (12 x 12), lam (12), rp/rq/rc/rs (6 each) are
// shared-memory workspace.  T = float (mixed precision) stops at a relative
// off-diagonal mass of 1e-11 and forms every entry of the result and its
// mirror from the same products, so the result is exactly symmetric.  Every
// lane of the warp must call it.
template <typename T>
__device__ inline void warp_project_psd(T* A, T* V, T* lam, int* rp, int* rq, T* rc, T* rs, int n, int lane) {
  constexpr bool F32 = sizeof(T) == 4;
  const T rel_tol = F32 ? T(1e-11) : T(1e-30);
  for (int e = lane; e < 144; e += 32) V[e] = ((e / 12) == (e % 12)) ? T(1) : T(0);
  // Gershgorin: skip when diagonally dominant with non-negative diagonal
  bool dom = true;
  if (lane < n) {
    T off = T(0);
    for (int j = 0; j < n; ++j)
      if (j != lane) off += fabs(A[12 * lane + j]);
    dom = A[13 * lane] >= off;
  }
  if (__all_sync(0xffffffffu, dom)) return;
  __syncwarp();
  for (int sweep = 0; sweep < 20; ++sweep) {
    T off = T(0), tot = T(0);
    for (int e = lane; e < 144; e += 32) {
      int i = e / 12, j = e % 12;
      if (i < n && j < n) {
        T a2 = A[e] * A[e];
        tot += a2;
        if (i != j) off += a2;
      }
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if (off <= rel_tol * tot || tot == T(0)) break;
    for (int r = 0; r < n - 1; ++r) {
      if (lane < n / 2) {
        int k = lane;
        int pa = k, pb = n - 1 - k;
        int p = pa == 0 ? 0 : 1 + (pa - 1 + r) % (n - 1);
        int q = 1 + (pb - 1 + r) % (n - 1);
        if (p > q) { int t = p; p = q; q = t; }
        T apq = A[12 * p + q];
        T c = T(1), sn = T(0);
        if (apq != T(0)) {
          T theta = (A[12 * q + q] - A[12 * p + p]) / (T(2) * apq);
          T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
          c = T(1) / sqrt(t * t + T(1));
          sn = t * c;
        }
        rp[k] = p; rq[k] = q; rc[k] = c; rs[k] = sn;
      }
      __syncwarp();
      int items = (n / 2) * n;
      for (int it = lane; it < items; it += 32) {  // rows: A <- J^T A
        int k = it / n, j = it % n;
        int p = rp[k], q = rq[k];
        T c = rc[k], sn = rs[k];
        T apj = A[12 * p + j], aqj = A[12 * q + j];
        A[12 * p + j] = c * apj - sn * aqj;
        A[12 * q + j] = sn * apj + c * aqj;
      }
      __syncwarp();
      for (int it = lane; it < items; it += 32) {  // columns: A <- A J, V <- V J
        int k = it / n, i = it % n;
        int p = rp[k], q = rq[k];
        T c = rc[k], sn = rs[k];
        T aip = A[12 * i + p], aiq = A[12 * i + q];
        A[12 * i + p] = c * aip - sn * aiq;
        A[12 * i + q] = sn * aip + c * aiq;
        T vip = V[12 * i + p], viq = V[12 * i + q];
        V[12 * i + p] = c * vip - sn * viq;
        V[12 * i + q] = sn * vip + c * viq;
      }
      __syncwarp();
    }
  }
  // A <- V max(diag, 0) V^T (eigenvalues staged in shared memory)
  if (lane < n) lam[lane] = fmax(A[13 * lane], T(0));
  __syncwarp();
  T out[5] = {0, 0, 0, 0, 0};
  int cnt = 0;
  for (int e = lane; e < 144; e += 32, ++cnt) {
    int i = e / 12, j = e % 12;
    if (F32 && i > j) { int t = i; i = j; j = t; }
    T sacc = T(0);
    if (i < n && j < n)
      for (int k = 0; k < n; ++k) sacc += V[12 * i + k] * lam[k] * V[12 * j + k];
    out[cnt] = sacc;
  }
  __syncwarp();
  cnt = 0;
  for (int e = lane; e < 144; e += 32, ++cnt) A[e] = out[cnt];
  __syncwarp();
}

}  // namespace ipc
