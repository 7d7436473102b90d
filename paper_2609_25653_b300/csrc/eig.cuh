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

}  // namespace ipc
