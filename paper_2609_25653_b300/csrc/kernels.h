// Host-side launchers of the ipcsim kernels (declarations).
#pragma once
#include <cuda_runtime.h>
#include "bvh.cuh"
#include "common.cuh"

namespace ipc {

// Kernel launches issued by this library (all simulators, all threads).
extern unsigned long long g_kernel_launches;
inline void count_launch(int n = 1) { __atomic_fetch_add(&g_kernel_launches, (unsigned long long)n, __ATOMIC_RELAXED); }

struct PcgArgs {
  DevScene S;
  int n_nodes;
  const int* row;
  const int* col;
  const double* val;
  const int* rec;
  const int* n_pairs;
  int cap;
  const double* pairH;
  int n_fric;
  const int* f_ids;
  const double* f_w;
  const double* f_Hu;
  const double* Dinv;
  const double* b;
  double* x;
  double* r;
  double* z;
  double* p;
  double* y;
  double* s;        // Chronopoulos-Gear auxiliary direction (A p)
  double* partial;  // 5 * grid doubles
  double rtol;
  int max_iter;
  int* out;         // [iterations, status, FP64 residual replacements]
  double* res;      // [relative residual]
  // mixed precision: FP32 copies of the operator and preconditioner, FP32
  // search direction and preconditioned residual; x, r, y and all dot
  // products stay FP64, and the residual is replaced by b - A x with the FP64
  // operator when the FP32 iteration has converged.
  int fp32;
  const float* val32;
  const float* pairH32;
  const float* f_Hu32;
  const float* Dinv32;
  float* z32;
  float* p32;
};

// fem.cu
void launch_predict(cudaStream_t, const DevScene&, const double* z, const double* zd, double dt, const double* g,
                    double* z_t, double* z_tilde);
void launch_kin_targets(cudaStream_t, const DevScene&, const double* T, double* xk_hat, double* stitch_hat);
void launch_vertex_positions(cudaStream_t, const DevScene&, const double* z, const double* xk, double* xv);
void launch_vertex_disp(cudaStream_t, const DevScene&, const double* p, const double* pD, double* pv);
void launch_inertia(cudaStream_t, const DevScene&, const double* z, const double* z_tilde, double* g, double* E,
                    int want_grad);
void launch_elastic(cudaStream_t, const DevScene&, const double* xv, double scale, int mode, int project, double* g,
                    double* Hval, double* tetH, double* E);
void launch_stitch(cudaStream_t, const DevScene&, const double* xv, const double* stitch_hat, double k_c, double scale,
                   int mode, double* g, double* E);
void launch_abd_orth(cudaStream_t, const DevScene&, const double* z, double kappa_A, double scale, int mode, int project,
                     double* g, double* Hval, double* E);
void launch_trial(cudaStream_t, int ndof, int nk3, const double* z, const double* p, double alpha, double* z_out,
                  const double* xk, const double* pD, const double* xk_hat, double* xk_out);
void launch_velocity(cudaStream_t, int ndof, const double* z, const double* z_t, double inv_dt, double* zd);
void launch_pnorm(cudaStream_t, int ndof, const double* p, int nk3, const double* pD, unsigned long long* out);
void launch_sub(cudaStream_t, int n, const double* a, const double* b, double* o);

// contact.cu
void launch_barrier(cudaStream_t, int grid, const DevScene&, const double* xv, const int* rec, const int* n_dev, int cap,
                    double sh, double kappa, double scale, int mode, int project, double* g, double* pairH, double* Dc,
                    const double* pD, double* gdir, double* E, unsigned long long* min_s);
void launch_friction_lag(cudaStream_t, int grid, const DevScene&, const double* xv, const int* rec, const int* n_dev,
                         int cap, double sh, double kappa, int* f_ids, double* f_w, double* f_n, double* f_lam);
void launch_friction(cudaStream_t, const DevScene&, const double* xv, const double* xv_t, int n, const int* f_ids,
                     const double* f_w, const double* f_n, const double* f_lam, double mu, double eps, double scale,
                     int mode, double* g, double* f_Hu, double* Dc, const double* pD, double* gdir, double* E);

// cull.cu
void launch_cull_brute(cudaStream_t, const DevScene&, const double* xv, double sh, int* rec, double* rec_s, int* count,
                       int cap);
void launch_ccd_brute(cudaStream_t, const DevScene&, const double* xv, const double* pv, double s_frac, int max_iter,
                      unsigned long long* alpha_bits, int* n_cand);

// bvh.cu
cudaError_t bvh_alloc(Bvh& B, int n);
void bvh_free(Bvh& B);
void bvh_leaf_boxes(cudaStream_t, Bvh& B, const int* ids, int nvp, const double* xv, const double* pv, double pad);
void bvh_refit(cudaStream_t, Bvh& B);
void bvh_build(cudaStream_t, Bvh& B);
void launch_cull_bvh(cudaStream_t, const DevScene&, const double* xv, double sh, double pad, Bvh& tri, Bvh& edge,
                     int* rec, double* rec_s, int* count, int cap, int* err);
void launch_ccd_bvh(cudaStream_t, const DevScene&, const double* xv, const double* pv, double s_frac, int max_iter,
                    Bvh& tri, Bvh& edge, unsigned long long* alpha_bits, int* n_cand, int* err);
void bvh_rebuild(cudaStream_t, const DevScene&, const double* xv, double pad, Bvh& tri, Bvh& edge);
void launch_sweep_bvh(cudaStream_t, const DevScene&, const double* xv, const double* pv, double pad, double s_frac,
                      int max_iter, Bvh& tri, Bvh& edge, int* cand, int* n_cand, int ccap,
                      unsigned long long* alpha_bits, int* n_ccd, int* err);
void launch_filter_active(cudaStream_t, int grid, const DevScene&, const double* xv, double sh, const int* cand,
                          const int* n_cand, int ccap, int* rec, double* rec_s, int* count, int cap);

// adjoint.cu
void launch_theta_grad(cudaStream_t, const DevScene&, const double* xv, const double* lam, double scale, double* out);
void launch_mass_apply(cudaStream_t, const DevScene&, const double* lam, double dt, double* y, double* yd);
void launch_friction_apply(cudaStream_t, const DevScene&, int n, const int* f_ids, const double* f_w, const double* f_Hu,
                           const double* lam, double* y);
void launch_dot(cudaStream_t, int n, const double* a, const double* b, double* out);
void launch_axpy(cudaStream_t, int n, const double* x, double alpha, const double* y, double* out);

// pcg.cu
void launch_dinv(cudaStream_t, int n_nodes, const int* diag, const double* val, const double* Dc, double* Dinv);
void launch_rhs(cudaStream_t, int n, const double* g, const double* gdir, double* rhs);
int pcg_max_blocks(int threads);
constexpr int PCG_ROW_GROUP = 4;  // default threads per BSR row in the PCG's SpMV
// rowg: threads per BSR row in the SpMV (2, 4, 8 or 16)
cudaError_t launch_pcg(cudaStream_t, int grid, int threads, const PcgArgs& a, int rowg = 4);
int pcg_max_blocks_fp32(int threads);
void launch_to_float(cudaStream_t, size_t n, const double* src, float* dst, const int* n_dev = nullptr, int stride = 0);

// conservative-advancement iterations per CCD candidate
constexpr int ACCD_MAX_ITER = 10000;

}  // namespace ipc
